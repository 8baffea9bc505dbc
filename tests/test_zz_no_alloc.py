"""The allocation-free entry point pa_hash_static against pa_hash_batch.

pa_hash_static exists for callers that cannot call cudaMalloc (a device whose
memory another framework's allocator has reserved, a real-time distillation
loop that must not pay allocation latency or cudaFree's device-wide
synchronisation). It keeps all scratch in one static device array inside
libpa.so, so successive calls reuse -- and must fully re-initialise -- the same
memory. These tests call it twice in a row with different blocks and require
bit-identical final keys to the allocating path (pa_plan + pa_set_seed +
pa_hash_batch) for the same inputs. This file sorts last so that a run which
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_1809_07592_gb300 as pa
from paper_1809_07592_gb300 import inputs
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_07592_gb300 import build
    build.build()
    pa.lib()


def batch_path(n, m, dtype, seed_dev, keys_dev):
    plan = pa.Plan(n, m, dtype)
    plan.set_seed(seed_dev)
    out = plan.hash(keys_dev)
    torch.cuda.synchronize()
    res = to_host(out, (m + 63) // 64)
    plan.close()
    return res


def static_path(n, m, dtype, seed_dev, keys_dev):
    nkeys, kstride = keys_dev.shape
    ow = (m + 63) // 64
    ow += ow & 1
    out = torch.full((nkeys, ow), -1, dtype=torch.int64, device="cuda")
    margin = pa.pa_hash_static(n, m, dtype, seed_dev, keys_dev, nkeys, kstride, out, ow)
    torch.cuda.synchronize()
    return to_host(out, (m + 63) // 64), margin


@pytest.mark.parametrize("dtype", [pa.PA_FP32_GUARD, pa.PA_FP64, pa.PA_NTT64], ids=["fp32g", "fp64", "ntt64"])
def test_static_matches_batch_on_two_calls_in_a_row(dtype):
    # two different blocks back to back: the second call must not see the first call's scratch
    blocks = [(1 << 20, 1 << 18, 2, 31), (300001, 123457, 1, 32)]
    for n, m, nkeys, base in blocks:
        seed = inputs.bernoulli_bits(base, 1, n + m - 1)
        keys = inputs.batch_keys(n, nkeys, base_seed=base)
        sd = to_dev(seed)[0]
        kd = to_dev(keys)
        got, margin = static_path(n, m, dtype, sd, kd)
        exp = batch_path(n, m, dtype, sd, kd)
        np.testing.assert_array_equal(got, exp)
        assert 0.0 <= margin < 0.05


def test_static_rejects_sizes_beyond_its_scratch():
    n, m = 1 << 21, 2  # n + m - 1 > 2^21
    sd = torch.zeros(((n + m + 62) // 64 + 1) & ~1, dtype=torch.int64, device="cuda")
    kd = torch.zeros((1, n // 64), dtype=torch.int64, device="cuda")
    out = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(pa.PAError) as e:
        pa.pa_hash_static(n, m, pa.PA_FP64, sd, kd, 1, n // 64, out, 2)
    assert e.value.code == pa.PA_EUNSUPPORTED

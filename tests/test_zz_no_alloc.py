"""The allocation-free entry point pa_hash_static against pa_hash_batch and the CPU oracle.

pa_hash_static exists for callers that cannot call cudaMalloc (a device whose
memory another framework's allocator has reserved, a real-time distillation
loop that must not pay allocation latency or cudaFree's device-wide
synchronisation). It keeps all scratch in one static device array inside
libpa.so, so successive calls reuse -- and must fully re-initialise -- the same
memory. These tests call it twice in a row with different blocks and require
bit-identical final keys to the allocating path (pa_plan + pa_set_seed +
pa_hash_batch) and to the oracle for the same inputs, at the smallest and the
largest transform length the array holds, and through its guard's recomputation
in FP64 and NTT64. This file sorts last so that a run which stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_1809_07592_gb300 as pa
from oracle import oracle
from paper_1809_07592_gb300 import inputs
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

MODES = [pa.PA_FP32_GUARD, pa.PA_FP64, pa.PA_NTT64]
MODE_ID = {pa.PA_FP32_GUARD: "fp32g", pa.PA_FP64: "fp64", pa.PA_NTT64: "ntt64"}


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


# (n, m, keys, base seed): a 2^21 transform with a key pair, a lone key at another length,
# the smallest transform (2^12), and a key pair just under the array's 2^21 limit
BLOCKS = [(1 << 20, 1 << 18, 2, 31), (300001, 123457, 1, 32), (3000, 1000, 2, 33), (1_500_000, 597_152, 2, 34)]


@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
def test_static_matches_batch_on_two_calls_in_a_row(dtype):
    # different blocks back to back: no call may see an earlier call's scratch
    for n, m, nkeys, base in BLOCKS:
        assert n + m - 1 <= 1 << 21
        seed = inputs.bernoulli_bits(base, 1, n + m - 1)
        keys = inputs.batch_keys(n, nkeys, base_seed=base)
        sd = to_dev(seed)[0]
        kd = to_dev(keys)
        got, margin = static_path(n, m, dtype, sd, kd)
        exp = batch_path(n, m, dtype, sd, kd)
        np.testing.assert_array_equal(got, exp, err_msg=f"(n, m) = ({n}, {m}) vs pa_hash_batch")
        for k in range(nkeys):
            np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, seed, keys[k]),
                                          err_msg=f"(n, m) = ({n}, {m}) key {k} vs the oracle")
        assert 0.0 <= margin < 0.05


# PA_STATIC_GUARD between the FP32 and the FP64 margins stops the recomputation in FP64; below
# every margin it runs on to the exact transform (whose margin is 0)
@pytest.mark.parametrize("nkeys", [1, 2])
@pytest.mark.parametrize("dtype,guard,final_margin_zero", [(pa.PA_FP32_GUARD, "1e-6", False),
                                                           (pa.PA_FP32_GUARD, "-1", True),
                                                           (pa.PA_FP64, "-1", True)],
                         ids=["fp32-to-fp64", "fp32-to-ntt64", "fp64-to-ntt64"])
def test_static_guard_escalation(dtype, guard, final_margin_zero, nkeys, monkeypatch):
    monkeypatch.setenv("PA_STATIC_GUARD", guard)
    n, m = 200003, 70001
    seed = inputs.bernoulli_bits(40 + nkeys, 1, n + m - 1)
    keys = inputs.batch_keys(n, nkeys, base_seed=40 + nkeys)
    sd, kd = to_dev(seed)[0], to_dev(keys)
    for _ in range(2):  # twice in a row: the recomputation leaves the array reusable
        got, margin = static_path(n, m, dtype, sd, kd)
        for k in range(nkeys):
            np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, seed, keys[k]), err_msg=f"key {k}")
        if final_margin_zero:
            assert margin == 0.0
        else:
            assert 0.0 <= margin < 1e-6  # the FP64 margin, below the guard


def test_static_rejects_sizes_beyond_its_scratch():
    n, m = 1 << 21, 2  # n + m - 1 > 2^21
    sd = torch.zeros(((n + m + 62) // 64 + 1) & ~1, dtype=torch.int64, device="cuda")
    kd = torch.zeros((1, n // 64), dtype=torch.int64, device="cuda")
    out = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(pa.PAError) as e:
        pa.pa_hash_static(n, m, pa.PA_FP64, sd, kd, 1, n // 64, out, 2)
    assert e.value.code == pa.PA_EUNSUPPORTED

"""Modified Toeplitz hash [I_m, T'] (Section 2.2, Eq. 2-3) through the C ABI vs the oracle, bit for bit."""
import numpy as np
import pytest
import torch

import paper_1809_07592_gb300 as pa
from oracle import oracle
from paper_1809_07592_gb300 import inputs
from tests.gpu_util import sample_rows, to_dev, to_host, unpack_rows

pytestmark = pytest.mark.gpu

MODES = [pa.PA_FP32_GUARD, pa.PA_FP64, pa.PA_NTT64]
MODE_ID = {pa.PA_FP32_GUARD: "fp32g", pa.PA_FP64: "fp64", pa.PA_NTT64: "ntt64"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_07592_gb300 import build
    build.build()
    pa.lib()


def run(n, m, dtype, keys, seed, guard=None):
    plan = pa.Plan(n, m, dtype, modified=True)
    if guard is not None:
        pa.pa_plan_set_guard(plan.handle, guard)
    plan.set_seed(to_dev(seed)[0])
    out, (marg, mode, esc) = plan.hash(to_dev(keys), info=True)
    torch.cuda.synchronize()
    res = to_host(out, (m + 63) // 64)
    shape = plan.shape()
    plan.close()
    return res, np.array(marg), np.array(mode), esc, shape


# (n, m): tiny, word-misaligned key offsets m, tall Toeplitz blocks (m > n - m), DV-QKD-like sizes
SIZES = [(2, 1), (65, 64), (100, 37), (1000, 999), (5000, 1500), (65536, 6554), (100003, 40001),
         (200000, 150001)]


@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
@pytest.mark.parametrize("n,m", SIZES)
def test_modified_bit_exact(n, m, dtype):
    seed = inputs.bernoulli_bits(n + m, 1, n - 1)
    keys = inputs.batch_keys(n, 3, base_seed=n + m)
    got, marg, mode, esc, _ = run(n, m, dtype, keys, seed)
    for k in range(3):
        np.testing.assert_array_equal(got[k], oracle.modified_hash(n, m, seed, keys[k]), err_msg=f"key {k}")
    assert esc == 0 and (marg < 0.05).all()


@pytest.mark.parametrize("n,ratio", [(1 << 20, 0.1), (1 << 20, 0.5), (1_000_000, 0.6)])
def test_modified_dv_qkd_sizes(n, ratio):
    """64 keys sharing one seed; the transform covers n - 1 instead of n + m - 1."""
    m = int(ratio * n)
    seed = inputs.bernoulli_bits(1, 1, n - 1)
    keys = inputs.batch_keys(n, 64, base_seed=1)
    got, marg, mode, esc, shape = run(n, m, pa.PA_FP32_GUARD, keys, seed)
    std = pa.Plan(n, m if m <= n else n, pa.PA_FP32_GUARD)
    assert shape[0] <= std.shape()[0] and shape[0] >= n - 1
    std.close()
    assert esc == 0 and (marg < 0.05).all()
    rows = sample_rows(m, 150, seed=m)
    bits = unpack_rows(got[[0, 33, 63]], m)
    for j, k in enumerate([0, 33, 63]):
        np.testing.assert_array_equal(bits[j][rows.astype(np.int64)], oracle.modified_rows(n, m, seed, keys[k], rows))


def test_modified_forced_escalation():
    """Every key recomputed by the FP64 (modified) fallback plan: same bits."""
    n, m = 70001, 30011
    seed = inputs.bernoulli_bits(2, 1, n - 1)
    keys = inputs.batch_keys(n, 3, base_seed=2)
    got, marg, mode, esc, _ = run(n, m, pa.PA_FP32_GUARD, keys, seed, guard=-1.0)
    assert esc == 3 and (mode != pa.PA_FP32_GUARD).all()
    for k in range(3):
        np.testing.assert_array_equal(got[k], oracle.modified_hash(n, m, seed, keys[k]))


def test_modified_host_buffers():
    n, m = 100003, 40001
    seed = inputs.bernoulli_bits(4, 1, n - 1)
    keys = inputs.batch_keys(n, 4, base_seed=4)
    kw, ow = (n + 63) // 64, (m + 63) // 64
    hk = torch.from_numpy(keys.view(np.int64).copy()).pin_memory()
    ho = torch.zeros((4, ow), dtype=torch.int64).pin_memory()
    p = pa.Plan(n, m, pa.PA_FP32_GUARD, modified=True)
    p.set_seed(to_dev(seed)[0])
    pa.pa_hash_host(p.handle, hk, 4, kw, ho, ow)
    p.close()
    got = ho.numpy().view(np.uint64)
    for k in range(4):
        np.testing.assert_array_equal(got[k], oracle.modified_hash(n, m, seed, keys[k]))


def test_modified_argument_errors():
    for n, m in [(10, 10), (10, 0), (1, 1)]:
        with pytest.raises(pa.PAError) as e:
            pa.Plan(n, m, pa.PA_FP32_GUARD, modified=True)
        assert e.value.code == pa.PA_EINVAL
    p = pa.Plan(1000, 300, pa.PA_FP32_GUARD, modified=True)
    with pytest.raises(pa.PAError) as e:  # the seed has n - 1 bits
        pa.pa_set_seed(p.handle, to_dev(inputs.bernoulli_bits(0, 1, 1299))[0], 1299)
    assert e.value.code == pa.PA_EINVAL
    p.close()


@pytest.mark.parametrize("dtype", [pa.PA_FP32_GUARD, pa.PA_FP64], ids=["fp32g", "fp64"])
@pytest.mark.parametrize("n,m", [(100, 37), (65536, 6554), (100003, 40001)])
def test_modified_single_key(n, m, dtype):
    """A lone key of the modified hash (half-length form with the key bit offset m)."""
    seed = inputs.bernoulli_bits(n, 3, n - 1)
    key = inputs.batch_keys(n, 1, base_seed=n)
    got, marg, mode, esc, _ = run(n, m, dtype, key, seed)
    np.testing.assert_array_equal(got[0], oracle.modified_hash(n, m, seed, key[0]))
    assert esc == 0 and marg[0] < 0.05

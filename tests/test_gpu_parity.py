"""CUDA path vs the CPU oracle, bit for bit, through the C ABI (libpa.so)."""
import numpy as np
import pytest
import torch

import paper_1809_07592_gb300 as pa
from oracle import oracle
from paper_1809_07592_gb300 import inputs
from tests.gpu_util import cover_rows, sample_rows, to_dev, to_host, unpack_rows

pytestmark = pytest.mark.gpu

MODES = [pa.PA_FP32_GUARD, pa.PA_FP64, pa.PA_NTT64]
MODE_ID = {pa.PA_FP32_GUARD: "fp32g", pa.PA_FP64: "fp64", pa.PA_NTT64: "ntt64"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_07592_gb300 import build
    build.build()
    pa.lib()


def run(n, m, dtype, keys_np, seed_np, info=True, guard=None):
    plan = pa.Plan(n, m, dtype)
    if guard is not None:
        pa.pa_plan_set_guard(plan.handle, guard)
    plan.set_seed(to_dev(seed_np)[0])
    keys = to_dev(keys_np)
    out, (marg, mode, esc) = plan.hash(keys, info=True)
    torch.cuda.synchronize()
    res = to_host(out, (m + 63) // 64)
    shape = plan.shape()
    plan.close()
    return res, np.array(marg), np.array(mode), esc, shape


# (n, m): tiny, ragged word tails, several tiles, the smallest and the two-level sizes
SMALL = [(1, 1), (2, 1), (63, 17), (64, 64), (65, 3), (1000, 999), (4095, 1), (5000, 1500), (20000, 20000),
         (65536, 6554), (131072, 32768), (100003, 40001), (300000, 30000)]


@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
@pytest.mark.parametrize("n,m", SMALL)
def test_single_key_bit_exact(n, m, dtype):
    key, seed = inputs.block_inputs(n, m, base_seed=n * 7 + m)
    got, marg, mode, esc, _ = run(n, m, dtype, key[None, :], seed)
    exp = oracle.toeplitz_hash(n, m, seed, key)
    np.testing.assert_array_equal(got[0], exp)
    assert marg[0] < 0.05 and esc == 0 and mode[0] == dtype


@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
@pytest.mark.parametrize("nkeys", [1, 2, 3, 7, 16])
def test_shared_seed_batch(nkeys, dtype):
    n, m = 40000, 9000
    seed = inputs.bernoulli_bits(5, 1, n + m - 1)
    keys = inputs.batch_keys(n, nkeys, base_seed=5)
    got, marg, mode, esc, _ = run(n, m, dtype, keys, seed)
    for k in range(nkeys):
        np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, seed, keys[k]), err_msg=f"key {k}")
    assert esc == 0 and (marg < 0.05).all()


def test_tail_bits_ignored_and_output_tail_zero():
    n, m = 1000, 700
    key, seed = inputs.block_inputs(n, m, base_seed=3)
    k2, s2 = key.copy(), seed.copy()
    k2[-1] |= np.uint64(0xFFFFFFFFFFFFFFFF) << np.uint64(n % 64)
    s2[-1] |= np.uint64(0xFFFFFFFFFFFFFFFF) << np.uint64((n + m - 1) % 64)
    exp = oracle.toeplitz_hash(n, m, seed, key)
    for dtype in MODES:
        plan = pa.Plan(n, m, dtype)
        plan.set_seed(to_dev(s2)[0])
        keys = to_dev(np.stack([k2, k2]), stride=20)
        out = torch.full((2, 16), -1, dtype=torch.int64, device="cuda")  # padding words must stay untouched
        plan.hash(keys, out=out)
        torch.cuda.synchronize()
        o = out.cpu().numpy().view(np.uint64)
        nw = (m + 63) // 64
        for k in range(2):
            np.testing.assert_array_equal(o[k, :nw], exp)
            assert int(o[k, nw - 1]) >> (m % 64) == 0
            assert (o[k, nw:] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
        plan.close()


def test_fp64_escalates_to_ntt():
    """FP64 keys that fail the guard are recomputed with the exact transform."""
    n, m = 20000, 7000
    seed = inputs.bernoulli_bits(12, 1, n + m - 1)
    keys = inputs.batch_keys(n, 2, base_seed=12)
    got, marg, mode, esc, _ = run(n, m, pa.PA_FP64, keys, seed, guard=-1.0)
    assert esc == 2 and (mode == pa.PA_NTT64).all() and (marg == 0).all()
    for k in range(2):
        np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, seed, keys[k]))


def test_forced_escalation_keeps_bits():
    """Guard threshold below every margin: each key goes through the FP64 recomputation."""
    n, m = 30000, 12000
    seed = inputs.bernoulli_bits(9, 1, n + m - 1)
    keys = inputs.batch_keys(n, 3, base_seed=9)
    got, marg, mode, esc, _ = run(n, m, pa.PA_FP32_GUARD, keys, seed, guard=-1.0)
    assert esc == 3 and (mode == pa.PA_FP64).all()
    for k in range(3):
        np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, seed, keys[k]))


@pytest.mark.parametrize("n,m", [(1 << 20, 1 << 18), (1 << 23, 1 << 21)])
def test_adversarial_all_ones_escalates_or_exact(n, m):
    """All-ones key and seed make |w| ~ n/2. FP32 must either resolve it (margin <= 0.25) or hand the
    key to FP64; past |w| = 2^21 it cannot resolve parity at all and must escalate."""
    ones_k = inputs.mask_tail(np.full((n + 63) // 64, 0xFFFFFFFFFFFFFFFF, dtype=np.uint64), n)
    ones_s = inputs.mask_tail(np.full((n + m + 62) // 64, 0xFFFFFFFFFFFFFFFF, dtype=np.uint64), n + m - 1)
    rnd = inputs.bernoulli_bits(1, 2, n)
    keys = np.stack([ones_k, rnd])
    got, marg, mode, esc, _ = run(n, m, pa.PA_FP32_GUARD, keys, ones_s)
    if n // 2 >= (1 << 21):
        assert mode[0] == pa.PA_FP64 and esc >= 1
    else:
        assert (mode[0] == pa.PA_FP64 and esc >= 1) or (mode[0] == pa.PA_FP32_GUARD and marg[0] <= 0.25)
    rows = sample_rows(m, 100)
    for k in range(2):
        exp = oracle.toeplitz_rows(n, m, ones_s, keys[k], rows)
        np.testing.assert_array_equal(unpack_rows(got, m)[k][rows.astype(np.int64)], exp)
    # all-ones seed: every output bit is the key's popcount parity
    assert (unpack_rows(got, m)[0] == (n & 1)).all()


@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
def test_result_independent_of_batch_mates(dtype):
    """A key's bits do not depend on the key sharing its complex transform."""
    n, m = 50000, 20000
    seed = inputs.bernoulli_bits(4, 1, n + m - 1)
    keys = inputs.batch_keys(n, 4, base_seed=4)
    alone, *_ = run(n, m, dtype, keys[1:2], seed)
    mixed, *_ = run(n, m, dtype, keys, seed)
    np.testing.assert_array_equal(alone[0], mixed[1])


@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
def test_every_pass_length(dtype):
    """Walk L = 2^12 .. 2^22 so every two-level split and kernel instance runs once."""
    for lgL in range(12, 23):
        n = (1 << (lgL - 1)) + 17
        m = max(1, (1 << lgL) - n - 5) if (1 << lgL) - n > 6 else 1
        key, seed = inputs.block_inputs(n, m, base_seed=lgL)
        got, marg, *_ , shape = run(n, m, dtype, key[None, :], seed)
        assert shape[0] == 1 << lgL
        rows = sample_rows(m, 300, seed=lgL)
        exp = oracle.toeplitz_rows(n, m, seed, key, rows)
        np.testing.assert_array_equal(unpack_rows(got, m)[0][rows.astype(np.int64)], exp, err_msg=f"lgL={lgL}")


@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
def test_three_level_plan(dtype):
    """Sizes beyond one CTA's innermost transform use the three-pass split."""
    lgL = 25 if dtype == pa.PA_FP32_GUARD else 24  # FP64 and NTT64 split earlier (wider elements)
    n = (1 << (lgL - 1)) + 1000
    m = (1 << (lgL - 2)) - 3
    key, seed = inputs.block_inputs(n, m, base_seed=77)
    got, marg, mode, esc, shape = run(n, m, dtype, key[None, :], seed)
    assert shape[3] > 1
    rows = cover_rows(m, shape)
    exp = oracle.toeplitz_rows(n, m, seed, key, rows)
    np.testing.assert_array_equal(unpack_rows(got, m)[0][rows.astype(np.int64)], exp)
    assert marg[0] < 0.1


@pytest.mark.parametrize("n", [1_000_000, 1 << 20])
@pytest.mark.parametrize("ratio", [0.1, 0.25, 0.5])
def test_dv_qkd_block_64_keys(n, ratio):
    """64 keys sharing one seed at the DV-QKD block sizes, FP32-guarded: the first and the last key
    (the real part of the first transform, the imaginary part of the last) whole vs the oracle,
    three more keys on rows that cover every digit of the plan's split."""
    m = int(ratio * n)
    seed = inputs.bernoulli_bits(0, 1, n + m - 1)
    keys = inputs.batch_keys(n, 64, base_seed=0)
    got, marg, mode, esc, shape = run(n, m, pa.PA_FP32_GUARD, keys, seed)
    assert esc == 0 and (marg < 0.05).all()
    for k in (0, 63):
        np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, seed, keys[k]), err_msg=f"key {k}")
    bits = unpack_rows(got[[1, 31, 62]], m)
    rows = cover_rows(m, shape, count=8192)
    for j, k in enumerate([1, 31, 62]):
        exp = oracle.toeplitz_rows(n, m, seed, keys[k], rows)
        np.testing.assert_array_equal(bits[j][rows.astype(np.int64)], exp, err_msg=f"key {k}")


def test_argument_errors():
    with pytest.raises(pa.PAError):
        pa.pa_plan(10, 11, pa.PA_FP64)  # m > n
    with pytest.raises(pa.PAError):
        pa.pa_plan(0, 0, pa.PA_FP64)
    plan = pa.Plan(1000, 100, pa.PA_FP32_GUARD)
    keys = torch.zeros((2, 16), dtype=torch.int64, device="cuda")
    out = torch.zeros((2, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(pa.PAError) as e:
        plan.hash(keys, out=out)
    assert e.value.code == pa.PA_ENOSEED
    seed = torch.zeros(18, dtype=torch.int64, device="cuda")
    with pytest.raises(pa.PAError) as e:
        pa.pa_set_seed(plan.handle, seed, 1000)  # wrong seed length
    assert e.value.code == pa.PA_EINVAL
    plan.set_seed(seed)
    with pytest.raises(pa.PAError) as e:
        pa.pa_hash_batch(plan.handle, keys, 2, 15, out, 2)  # odd stride
    assert e.value.code == pa.PA_EINVAL
    with pytest.raises(pa.PAError) as e:
        pa.pa_hash_batch(plan.handle, keys[:, 1:], 2, 16, out, 2)  # misaligned
    assert e.value.code == pa.PA_EINVAL
    plan.close()


@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
def test_long_block_2p27(dtype):
    """The long single block: n = 2^27, m = 2^24, transform length 2^28, seed spectrum resident."""
    n, m = 1 << 27, 1 << 24
    key, seed = inputs.block_inputs(n, m, base_seed=0)
    got, marg, mode, esc, shape = run(n, m, dtype, key[None, :], seed)
    assert n + m - 1 <= shape[0] <= 1 << 28 and shape[3] > 1
    if dtype == pa.PA_NTT64:
        assert shape[0] == 1 << 28  # the exact transform keeps power-of-two lengths
    rows = cover_rows(m, shape)
    exp = oracle.toeplitz_rows(n, m, seed, key, rows)
    np.testing.assert_array_equal(unpack_rows(got, m)[0][rows.astype(np.int64)], exp)
    if dtype == pa.PA_FP32_GUARD:
        assert mode[0] in (pa.PA_FP32_GUARD, pa.PA_FP64)  # the guard may hand it to FP64
    assert marg[0] < 0.25


# (n, m) whose n+m-1 lands just below RO * 2^k: every odd factor and a range of innermost lengths
SMOOTH = [(ro, k) for ro in (3, 5, 9) for k in (13, 15, 17, 19)]


@pytest.mark.parametrize("dtype", [pa.PA_FP32_GUARD, pa.PA_FP64], ids=["fp32g", "fp64"])
@pytest.mark.parametrize("ro,k", SMOOTH)
def test_smooth_lengths_bit_exact(ro, k, dtype):
    """Transform lengths 3, 5 or 9 times a power of two (odd-radix stage in the innermost pass)."""
    n, m = 2**k * ro * 2 // 3 + 7, 2**k * ro // 3 - 20  # n + m - 1 just below ro * 2^k
    key, seed = inputs.block_inputs(n, m, base_seed=n)
    keys = np.stack([key, inputs.bernoulli_bits(n, 9, n), inputs.bernoulli_bits(n, 10, n)])
    got, marg, mode, esc, shape = run(n, m, dtype, keys, seed)
    assert shape[0] == ro << k, shape
    for k in range(3):
        if n <= 200_000:
            np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, seed, keys[k]))
        else:
            rows = sample_rows(m, 150, seed=k)
            exp = oracle.toeplitz_rows(n, m, seed, keys[k], rows)
            np.testing.assert_array_equal(unpack_rows(got, m)[k][rows.astype(np.int64)], exp)
    assert esc == 0 and (marg < 0.1).all()


@pytest.mark.parametrize("dtype", [pa.PA_FP32_GUARD, pa.PA_FP64], ids=["fp32g", "fp64"])
def test_smooth_three_level(dtype):
    """An odd innermost length under a three-level split (n+m-1 just below 3 * 2^23)."""
    n, m = (1 << 24) - 5, (1 << 23) - 11
    key, seed = inputs.block_inputs(n, m, base_seed=31)
    got, marg, mode, esc, shape = run(n, m, dtype, key[None, :], seed)
    assert shape[0] == 3 << 23 and shape[3] > 1
    rows = cover_rows(m, shape)
    exp = oracle.toeplitz_rows(n, m, seed, key, rows)
    np.testing.assert_array_equal(unpack_rows(got, m)[0][rows.astype(np.int64)], exp)


@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
@pytest.mark.parametrize("n,m", [(1 << 20, 1 << 18), (1_000_000, 100_000), (1_000_000, 500_000), (5000, 1500)])
def test_every_split_bit_exact(n, m, dtype):
    """Every pass split the autotuner can pick gives the same bits; sampled rows match the oracle."""
    seed = inputs.bernoulli_bits(11, 1, n + m - 1)
    keys = inputs.batch_keys(n, 3, base_seed=11)
    splits = pa.pa_plan_splits(n, m, dtype)
    rows = sample_rows(m, 120, seed=m)
    exp = [oracle.toeplitz_rows(n, m, seed, keys[k], rows) for k in range(3)]
    first = None
    for split in splits:
        plan = pa.Plan(n, m, dtype, split=split)
        assert tuple(plan.shape()[1:]) == tuple(split)
        plan.set_seed(to_dev(seed)[0])
        out, (marg, mode, esc) = plan.hash(to_dev(keys), info=True)
        torch.cuda.synchronize()
        got = to_host(out, (m + 63) // 64)
        plan.close()
        assert esc == 0 and max(marg) < 0.1, (split, marg)
        bits = unpack_rows(got, m)
        for k in range(3):
            np.testing.assert_array_equal(bits[k][rows.astype(np.int64)], exp[k], err_msg=f"split {split} key {k}")
        if first is None:
            first = got
        else:
            np.testing.assert_array_equal(got, first, err_msg=f"split {split}")
    tuned = pa.Plan(n, m, dtype)
    assert tuple(tuned.shape()[1:]) in {tuple(s) for s in splits}
    tuned.close()


def test_forced_split_rejects_unlisted():
    with pytest.raises(pa.PAError) as e:
        pa.Plan(1 << 20, 1 << 18, pa.PA_FP32_GUARD, split=(64, 64, 1))
    assert e.value.code == pa.PA_EINVAL


def test_async_issue_then_finish_matches_sync():
    """Batches of three plans issued back to back, then finished: same bits as pa_hash_batch."""
    cases = [(40000, 9000), (100003, 40001), (1 << 20, 1 << 18)]
    plans, bufs = [], []
    for i, (n, m) in enumerate(cases):
        seed = inputs.bernoulli_bits(21 + i, 1, n + m - 1)
        keys = inputs.batch_keys(n, 5, base_seed=21 + i)
        p = pa.Plan(n, m, pa.PA_FP32_GUARD)
        p.set_seed(to_dev(seed)[0])
        dk = to_dev(keys)
        ref = to_host(p.hash(dk), (m + 63) // 64)
        ow = (m + 63) // 64 + ((m + 63) // 64 & 1)
        out = torch.full((5, ow), -1, dtype=torch.int64, device="cuda")
        plans.append(p)
        bufs.append((dk, out, ref, n, m, seed, keys))
    for p, (dk, out, *_rest) in zip(plans, bufs):
        pa.pa_hash_batch_async(p.handle, dk, 5, dk.shape[1], out, out.shape[1])
    with pytest.raises(pa.PAError) as e:  # one batch in flight per plan
        pa.pa_hash_batch_async(plans[0].handle, bufs[0][0], 5, bufs[0][0].shape[1], bufs[0][1], bufs[0][1].shape[1])
    assert e.value.code == pa.PA_EAGAIN
    for p, (dk, out, ref, n, m, seed, keys) in zip(plans, bufs):
        marg, mode, esc = pa.pa_batch_finish(p.handle, 5, info=True)
        assert esc == 0 and max(marg) < 0.05
        got = to_host(out, (m + 63) // 64)
        np.testing.assert_array_equal(got, ref)
        rows = sample_rows(m, 50, seed=1)
        np.testing.assert_array_equal(unpack_rows(got, m)[4][rows.astype(np.int64)],
                                      oracle.toeplitz_rows(n, m, seed, keys[4], rows))
    with pytest.raises(pa.PAError) as e:  # nothing issued
        pa.pa_batch_finish(plans[0].handle)
    assert e.value.code == pa.PA_EINVAL
    for p in plans:
        p.close()


def test_async_forced_escalation():
    """The guard step of an issued batch escalates like pa_hash_batch (threshold -1: every key)."""
    n, m = 65536, 6554
    seed = inputs.bernoulli_bits(4, 1, n + m - 1)
    keys = inputs.batch_keys(n, 3, base_seed=4)
    p = pa.Plan(n, m, pa.PA_FP32_GUARD)
    pa.pa_plan_set_guard(p.handle, -1.0)
    p.set_seed(to_dev(seed)[0])
    dk = to_dev(keys)
    out = torch.empty((3, 104), dtype=torch.int64, device="cuda")
    pa.pa_hash_batch_async(p.handle, dk, 3, dk.shape[1], out, out.shape[1])
    marg, mode, esc = pa.pa_batch_finish(p.handle, 3, info=True)
    assert esc == 3 and all(md in (pa.PA_FP64, pa.PA_NTT64) for md in mode)
    got = to_host(out, (m + 63) // 64)
    for k in range(3):
        np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, seed, keys[k]))
    p.close()


def _host_rows(arr_u64, stride, pinned):
    """(nkeys, stride) int64 CPU tensor holding arr_u64 rows (padding words = a marker)."""
    nk, nw = arr_u64.shape
    t = torch.full((nk, stride), 0x5A5A, dtype=torch.int64)
    if pinned:
        t = t.pin_memory()
    t[:, :nw] = torch.from_numpy(arr_u64.view(np.int64))
    return t


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
def test_host_buffers_bit_exact(dtype, pinned):
    """Keys from host memory, final keys back to host memory (odd strides, padding untouched)."""
    n, m, nk = 100003, 40001, 5
    seed = inputs.bernoulli_bits(31, 1, n + m - 1)
    keys = inputs.batch_keys(n, nk, base_seed=31)
    kw, ow = (n + 63) // 64, (m + 63) // 64
    hk = _host_rows(keys, kw + 3, pinned)
    ho = torch.full((nk, ow + 5), 0x77, dtype=torch.int64)
    if pinned:
        ho = ho.pin_memory()
    p = pa.Plan(n, m, dtype)
    p.set_seed(to_dev(seed)[0])
    marg, mode, esc = pa.pa_hash_host(p.handle, hk, nk, hk.shape[1], ho, ho.shape[1], info=True)
    p.close()
    got = ho.numpy().view(np.uint64)
    for k in range(nk):
        np.testing.assert_array_equal(got[k, :ow], oracle.toeplitz_hash(n, m, seed, keys[k]), err_msg=f"key {k}")
    assert (ho.numpy()[:, ow:] == 0x77).all()  # words past each row untouched
    assert esc == 0 and max(marg) < 0.05


def test_host_buffers_escalation_rewrites_rows():
    """A key recomputed by the guard is rewritten in host memory."""
    n, m, nk = 65536, 6554, 3
    seed = inputs.bernoulli_bits(8, 1, n + m - 1)
    keys = inputs.batch_keys(n, nk, base_seed=8)
    hk = _host_rows(keys, (n + 63) // 64, True)
    ow = (m + 63) // 64
    ho = torch.zeros((nk, ow), dtype=torch.int64).pin_memory()
    p = pa.Plan(n, m, pa.PA_FP32_GUARD)
    pa.pa_plan_set_guard(p.handle, -1.0)
    p.set_seed(to_dev(seed)[0])
    marg, mode, esc = pa.pa_hash_host(p.handle, hk, nk, hk.shape[1], ho, ow, info=True)
    p.close()
    assert esc == nk
    got = ho.numpy().view(np.uint64)
    for k in range(nk):
        np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, seed, keys[k]))


def test_host_buffers_three_plans_pipelined():
    """Host batches of three plans issued back to back (copies overlap compute), then finished."""
    cases = [(40000, 9000), (1 << 20, 1 << 18), (100003, 40001)]
    plans, bufs = [], []
    for i, (n, m) in enumerate(cases):
        seed = inputs.bernoulli_bits(50 + i, 1, n + m - 1)
        keys = inputs.batch_keys(n, 4, base_seed=50 + i)
        p = pa.Plan(n, m, pa.PA_FP32_GUARD)
        p.set_seed(to_dev(seed)[0])
        hk = _host_rows(keys, (n + 63) // 64, True)
        ho = torch.zeros((4, (m + 63) // 64), dtype=torch.int64).pin_memory()
        plans.append(p)
        bufs.append((hk, ho, n, m, seed, keys))
    for _ in range(2):  # twice: the second round reuses the staging rows
        for p, (hk, ho, *_r) in zip(plans, bufs):
            ho.zero_()
            pa.pa_hash_host_async(p.handle, hk, 4, hk.shape[1], ho, ho.shape[1])
        for p, (hk, ho, n, m, seed, keys) in zip(plans, bufs):
            pa.pa_batch_finish(p.handle)
            got = ho.numpy().view(np.uint64)
            rows = sample_rows(m, 60, seed=2)
            for k in (0, 3):
                np.testing.assert_array_equal(unpack_rows(got, m)[k][rows.astype(np.int64)],
                                              oracle.toeplitz_rows(n, m, seed, keys[k], rows))
    for p in plans:
        p.close()


@pytest.mark.parametrize("dtype", [pa.PA_FP32_GUARD, pa.PA_FP64], ids=["fp32g", "fp64"])
@pytest.mark.parametrize("n,m", [(1, 1), (63, 17), (4095, 1), (5000, 1500), (131072, 32768), (100003, 40001),
                                 (1_000_000, 500_000), ((1 << 23) + 5, (1 << 21) - 3)])
def test_single_key_half_length_form(n, m, dtype):
    """A lone key runs in the half-length transform (bins k, N-k split against seed tables):
    same bits as the key paired with another one, and as the oracle."""
    seed = inputs.bernoulli_bits(n + 3, 1, n + m - 1)
    keys = inputs.batch_keys(n, 2, base_seed=n + 3)
    plan = pa.Plan(n, m, dtype)
    plan.set_seed(to_dev(seed)[0])
    one, (marg1, mode1, esc1) = plan.hash(to_dev(keys[:1]), info=True)
    two = plan.hash(to_dev(keys))
    torch.cuda.synchronize()
    plan.close()
    w = (m + 63) // 64
    one, two = to_host(one, w), to_host(two, w)
    np.testing.assert_array_equal(one[0], two[0])
    assert esc1 == 0 and marg1[0] < 0.05
    if n <= 200_000:
        np.testing.assert_array_equal(one[0], oracle.toeplitz_hash(n, m, seed, keys[0]))
    else:
        rows = sample_rows(m, 120, seed=n)
        np.testing.assert_array_equal(unpack_rows(one, m)[0][rows.astype(np.int64)],
                                      oracle.toeplitz_rows(n, m, seed, keys[0], rows))


@pytest.mark.parametrize("dtype", [pa.PA_FP64, pa.PA_NTT64], ids=["fp64", "ntt64"])
def test_plan_on_several_streams(dtype):
    """One plan driven from three streams with no host wait in between (FP64 and NTT64 return
    right after issuing): batches, and a seed change between them, run in issue order."""
    n, m, nk = 1 << 20, 1 << 18, 6
    seeds = [inputs.bernoulli_bits(90 + s, 1, n + m - 1) for s in range(2)]
    keys = [inputs.batch_keys(n, nk, base_seed=90 + b) for b in range(4)]
    plan = pa.Plan(n, m, dtype)
    streams = [torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()]
    dseeds = [to_dev(s)[0] for s in seeds]
    dkeys = [to_dev(k) for k in keys]
    ow = (m + 63) // 64
    outs = [torch.full((nk, ow), -1, dtype=torch.int64, device="cuda") for _ in keys]
    torch.cuda.synchronize()
    plan.set_seed(dseeds[0], stream=streams[2])
    for b in range(4):
        if b == 2:
            plan.set_seed(dseeds[1], stream=streams[1])
        st = streams[b % 3]
        pa.pa_hash_batch(plan.handle, dkeys[b], nk, dkeys[b].shape[1], outs[b], ow, st)
    torch.cuda.synchronize()
    plan.close()
    rows = sample_rows(m, 80, seed=9)
    for b in range(4):
        seed = seeds[0] if b < 2 else seeds[1]
        got = unpack_rows(to_host(outs[b], ow), m)
        for k in (0, nk - 1):
            np.testing.assert_array_equal(got[k][rows.astype(np.int64)],
                                          oracle.toeplitz_rows(n, m, seed, keys[b][k], rows))


@pytest.mark.parametrize("host", [False, True], ids=["device", "host"])
def test_dv_qkd_step_on_two_streams(host):
    """The benchmark's step as it is timed: the six DV-QKD batches (64 keys each, one seed per
    (n, m)) issued back to back alternating between two streams, then finished; device-resident
    buffers, or host buffers through pa_hash_host_async. Keys 0 and 63 of every batch whole vs the
    oracle, sampled rows of key 33, and every key equal to the same batch run alone."""
    nk = 64
    sides = [torch.cuda.Stream(), torch.cuda.Stream()]
    cases = []
    for n in (1_000_000, 1 << 20):
        for ratio in (0.1, 0.25, 0.5):
            m = int(ratio * n)
            seed = inputs.bernoulli_bits(0, inputs.STREAM_SEED, n + m - 1)
            keys = inputs.batch_keys(n, nk, base_seed=0)
            p = pa.Plan(n, m, pa.PA_FP32_GUARD)
            p.set_seed(to_dev(seed)[0])
            kw = keys.shape[1] + (keys.shape[1] & 1)
            ow = (m + 63) // 64 + ((m + 63) // 64 & 1)
            if host:
                ki = _host_rows(keys, kw, True)
                out = torch.zeros((nk, ow), dtype=torch.int64).pin_memory()
            else:
                ki = to_dev(keys, kw)
                out = torch.full((nk, ow), -1, dtype=torch.int64, device="cuda")
            cases.append(dict(n=n, m=m, seed=seed, keys=keys, plan=p, ki=ki, out=out, kw=kw, ow=ow))
    torch.cuda.synchronize()
    main = torch.cuda.current_stream()
    for sd in sides:
        sd.wait_stream(main)
    for i, c in enumerate(cases):
        issue = pa.pa_hash_host_async if host else pa.pa_hash_batch_async
        issue(c["plan"].handle, c["ki"], nk, c["kw"], c["out"], c["ow"], sides[i % 2])
    for c in cases:
        marg, mode, esc = pa.pa_batch_finish(c["plan"].handle, nk, info=True)
        assert esc == 0 and max(marg) < 0.05
    for sd in sides:
        main.wait_stream(sd)
    torch.cuda.synchronize()
    for c in cases:
        n, m = c["n"], c["m"]
        w = (m + 63) // 64
        got = (c["out"].numpy() if host else c["out"].cpu().numpy()).view(np.uint64)[:, :w]
        alone = to_host(c["plan"].hash(to_dev(c["keys"], c["kw"])), w)
        np.testing.assert_array_equal(got, alone, err_msg=f"(n, m) = ({n}, {m}): two-stream step vs alone")
        for k in (0, 63):
            np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(n, m, c["seed"], c["keys"][k]),
                                          err_msg=f"(n, m) = ({n}, {m}), key {k}")
        rows = sample_rows(m, 300, seed=m)
        np.testing.assert_array_equal(unpack_rows(got[[33]], m)[0][rows.astype(np.int64)],
                                      oracle.toeplitz_rows(n, m, c["seed"], c["keys"][33], rows),
                                      err_msg=f"(n, m) = ({n}, {m}), key 33")
        c["plan"].close()


@pytest.mark.parametrize("modified", [False, True], ids=["standard", "modified"])
@pytest.mark.parametrize("n,m", [(1 << 20, 104_857), (1 << 20, 1 << 18), (1_000_000, 500_000), (100_003, 40_001)])
def test_staged_last_pass_bit_exact(n, m, modified):
    """The TMA-staged last pass (pa_plan_set_staged) gives the same bits as the plain one on every
    split; keys 0 and the last whole vs the oracle (odd key count: the lone key keeps its own form)."""
    nk = 9
    seed = inputs.bernoulli_bits(70 + m, 1, (n - 1) if modified else (n + m - 1))
    keys = inputs.batch_keys(n, nk, base_seed=70 + m)
    ow = (m + 63) // 64
    splits = pa.pa_plan_splits(n - m if modified else n, m, pa.PA_FP32_GUARD) if not modified else [None]
    for split in splits:
        outs = []
        for staged in (False, True):
            p = pa.Plan(n, m, pa.PA_FP32_GUARD, split=split, modified=modified)
            pa.pa_plan_set_staged(p.handle, staged)
            p.set_seed(to_dev(seed)[0])
            out, (marg, mode, esc) = p.hash(to_dev(keys), info=True)
            torch.cuda.synchronize()
            outs.append(to_host(out, ow))
            assert esc == 0 and max(marg) < 0.05
            p.close()
        np.testing.assert_array_equal(outs[1], outs[0], err_msg=f"split {split}: staged vs plain")
    ref = oracle.modified_hash if modified else oracle.toeplitz_hash
    for k in (0, nk - 1):
        np.testing.assert_array_equal(outs[1][k], ref(n, m, seed, keys[k]), err_msg=f"key {k}")

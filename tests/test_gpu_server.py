"""Serving loop: continuous batching, admission by HBM footprint, results vs the oracle."""
import time

import numpy as np
import pytest
import torch

import paper_1809_07592_gb300 as pa
from oracle import oracle
from paper_1809_07592_gb300 import inputs
from tests.gpu_util import sample_rows, to_dev, unpack_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_07592_gb300 import build
    build.build()
    pa.lib()


def make_block(n, m, base, b):
    k = inputs.bernoulli_bits(base, 2 * b + 2, n)
    s = inputs.bernoulli_bits(base, 2 * b + 3, n + m - 1)
    ow = (m + 63) // 64
    out = torch.full((ow + (ow & 1),), -1, dtype=torch.int64, device="cuda")
    return dict(n=n, m=m, k=k, s=s, kd=to_dev(k)[0], sd=to_dev(s)[0], out=out)


def check(blk, nrows=150):
    n, m = blk["n"], blk["m"]
    got = blk["out"].cpu().numpy().view(np.uint64)[: (m + 63) // 64]
    if n <= 300_000:
        np.testing.assert_array_equal(got, oracle.toeplitz_hash(n, m, blk["s"], blk["k"]))
    else:
        rows = sample_rows(m, nrows, seed=n)
        exp = oracle.toeplitz_rows(n, m, blk["s"], blk["k"], rows)
        np.testing.assert_array_equal(unpack_rows(got[None, :], m)[0][rows.astype(np.int64)], exp)


def submit_all(srv, blocks):
    return [pa.pa_submit(srv, b["n"], b["m"], b["kd"], b["sd"], b["out"]) for b in blocks]


def wait_all(srv, tickets, timeout_ms=60000):
    res = [pa.pa_wait(srv, t, timeout_ms) for t in tickets]
    torch.cuda.synchronize()
    return res


SIZES = [(1000, 500), (5000, 1500), (131072, 32768), (100003, 40001), (1 << 18, 1 << 16), (1_000_000, 250_000),
         (1 << 20, 1 << 19), (70000, 7000), (300000, 150000), (1 << 22, 1 << 20), (64, 64), (4095, 2000)]


@pytest.mark.parametrize("dtype", [pa.PA_FP32_GUARD, pa.PA_FP64], ids=["fp32g", "fp64"])
def test_server_results_bit_exact(dtype):
    blocks = [make_block(n, m, 21, b) for b, (n, m) in enumerate(SIZES)]
    srv = pa.pa_server_create(dtype=dtype, max_batch=5, streams=3)
    res = wait_all(srv, submit_all(srv, blocks))
    for r, b in zip(res, blocks):
        assert r.status == pa.PA_OK and r.margin < 0.05
        assert r.t_submit_ns <= r.t_admit_ns <= r.t_done_ns
        check(b)
    st = pa.pa_server_stats(srv)
    assert st["completed"] == len(blocks) and st["inflight_bytes"] == 0
    pa.pa_server_destroy(srv)


def test_block_same_alone_and_in_the_mix():
    """Results do not depend on what else is in flight: bits equal alone and in a busy mix."""
    blocks = [make_block(n, m, 22, b) for b, (n, m) in enumerate(SIZES)]
    srv = pa.pa_server_create(dtype=pa.PA_FP32_GUARD, max_batch=4, streams=4)
    wait_all(srv, submit_all(srv, blocks))
    mixed = [b["out"].clone() for b in blocks]
    for i, b in enumerate(blocks):
        b["out"].fill_(-1)
        wait_all(srv, [pa.pa_submit(srv, b["n"], b["m"], b["kd"], b["sd"], b["out"])])
        assert torch.equal(b["out"], mixed[i]), f"block {i} differs alone vs in the mix"
    pa.pa_server_destroy(srv)


def test_admission_cap_is_respected():
    blocks = [make_block(1 << 20, 1 << 18, 23, b) for b in range(12)]
    one = 3 * (1 << 21) * 8 // 2 + 4096  # about one block's scratch at L = 2^21, FP32
    srv = pa.pa_server_create(hbm_cap_bytes=2 * one, dtype=pa.PA_FP32_GUARD, max_batch=8, streams=4)
    res = wait_all(srv, submit_all(srv, blocks))
    st = pa.pa_server_stats(srv)
    assert all(r.status == pa.PA_OK for r in res)
    assert 0 < st["peak_inflight_bytes"] <= 2 * one
    for b in blocks[:3]:
        check(b)
    pa.pa_server_destroy(srv)


def test_queue_full_and_wait_timeout():
    big = [make_block(1 << 24, 1 << 23, 24, b) for b in range(2)]
    cap = 3 * (1 << 25) * 16 // 2 + 4096  # one FP64 block of L = 2^25 at a time
    srv = pa.pa_server_create(hbm_cap_bytes=cap, dtype=pa.PA_FP64, max_queue=2, max_batch=1, streams=2)
    t0 = pa.pa_submit(srv, big[0]["n"], big[0]["m"], big[0]["kd"], big[0]["sd"], big[0]["out"])
    t1 = pa.pa_submit(srv, big[1]["n"], big[1]["m"], big[1]["kd"], big[1]["sd"], big[1]["out"])
    with pytest.raises(pa.PAError) as e:
        pa.pa_submit(srv, big[1]["n"], big[1]["m"], big[1]["kd"], big[1]["sd"], big[1]["out"])
    assert e.value.code == pa.PA_EAGAIN
    with pytest.raises(pa.PAError) as e:
        pa.pa_wait(srv, t1, 0)  # the second block cannot be done yet: it waits for the cap
    assert e.value.code == pa.PA_ETIMEOUT
    res = wait_all(srv, [t0, t1])
    assert all(r.status == pa.PA_OK for r in res)
    with pytest.raises(pa.PAError):
        pa.pa_poll(srv, t0)  # released after collection
    assert pa.pa_server_stats(srv)["rejected"] == 1
    pa.pa_server_destroy(srv)


def test_poisson_arrivals_short_run():
    """A short serving run with Poisson arrivals; every collected result is checked."""
    times, sizes = inputs.serving_requests(120, rate_per_s=2000.0, base_seed=3)
    blocks = [make_block(n, m, 25, b) for b, (n, m) in enumerate(sizes)]
    srv = pa.pa_server_create(dtype=pa.PA_FP32_GUARD)
    t0 = time.perf_counter()
    tickets = []
    for t, b in zip(times, blocks):
        while time.perf_counter() - t0 < t:
            pass
        tickets.append(pa.pa_submit(srv, b["n"], b["m"], b["kd"], b["sd"], b["out"]))
    res = wait_all(srv, tickets)
    lat = np.array([(r.t_done_ns - r.t_submit_ns) / 1e6 for r in res])
    assert all(r.status == pa.PA_OK for r in res) and np.isfinite(lat).all()
    for b in blocks[::10]:
        check(b, nrows=60)
    pa.pa_server_destroy(srv)

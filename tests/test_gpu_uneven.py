"""Uneven batches (blocks of different (n, m), each with its own seed) vs the CPU oracle."""
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


def device_blocks(sizes, data):
    blocks, outs = [], []
    for (n, m), (k, s) in zip(sizes, data):
        ow = (m + 63) // 64
        out = torch.full((ow + (ow & 1),), -1, dtype=torch.int64, device="cuda")
        kd, sd = to_dev(k)[0], to_dev(s)[0]
        blocks.append((n, m, kd, sd, out))
        outs.append(out)
    return blocks


def class_shape(h, n, m):
    """(L, L1, L2, L3) of the class that holds a block: the smallest class length >= n + m - 1
    (a block's class is the smallest smooth length that fits it, and every class length is smooth)."""
    fits = [c for c in pa.pa_uneven_classes(h) if c[0] >= n + m - 1]
    c = min(fits, key=lambda c: c[0])
    return (c[0], c[1], c[2], c[3])


def check_blocks(sizes, data, blocks, full_limit=400_000, nrows=200, h=None):
    """Blocks with n <= full_limit whole vs the oracle; larger ones on nrows rows (covering every digit
    of their class's split when the batch handle h is given, else sampled)."""
    for b, ((n, m), (k, s), blk) in enumerate(zip(sizes, data, blocks)):
        got = blk[4].cpu().numpy().view(np.uint64)[: (m + 63) // 64]
        if n <= full_limit:
            np.testing.assert_array_equal(got, oracle.toeplitz_hash(n, m, s, k), err_msg=f"block {b} n={n} m={m}")
        else:
            rows = cover_rows(m, class_shape(h, n, m), count=nrows) if h is not None else sample_rows(m, nrows, seed=b)
            exp = oracle.toeplitz_rows(n, m, s, k, rows)
            np.testing.assert_array_equal(unpack_rows(got[None, :], m)[0][rows.astype(np.int64)], exp,
                                          err_msg=f"block {b} n={n} m={m}")
        # tail bits of the last word are zero
        if m % 64:
            assert int(got[-1]) >> (m % 64) == 0


SMALL = [(1, 1), (100, 37), (1000, 999), (4095, 2000), (5000, 1500), (65536, 6554), (70000, 42000), (131072, 32768),
         (100003, 40001), (250000, 150000), (300000, 30000), (5001, 1501), (64, 64)]


@pytest.mark.parametrize("graph", [True, False], ids=["graph", "direct"])
@pytest.mark.parametrize("dtype", MODES, ids=MODE_ID.get)
def test_uneven_bit_exact(dtype, graph):
    data = [(inputs.bernoulli_bits(3, 2 * b + 2, n), inputs.bernoulli_bits(3, 2 * b + 3, n + m - 1))
            for b, (n, m) in enumerate(SMALL)]
    blocks = device_blocks(SMALL, data)
    h = pa.pa_uneven_create(blocks, dtype, use_graph=graph)
    marg, mode, esc = pa.pa_uneven_run(h, len(blocks), info=True)
    torch.cuda.synchronize()
    check_blocks(SMALL, data, blocks)
    assert esc == 0 and max(marg) < 0.05 and all(md == dtype for md in mode)
    classes = pa.pa_uneven_classes(h)
    assert sum(c[4] for c in classes) == len(SMALL)
    pa.pa_uneven_destroy(h)


@pytest.mark.parametrize("dtype", [pa.PA_FP32_GUARD, pa.PA_FP64], ids=["fp32g", "fp64"])
def test_uneven_three_level_class(dtype):
    sizes = [(1 << 23, 1 << 21), ((1 << 23) - 12345, 3 << 20), ((1 << 22) + 5, 1 << 22)]
    data = inputs.uneven_block_inputs(sizes, base_seed=5)
    blocks = device_blocks(sizes, data)
    h = pa.pa_uneven_create(blocks, dtype, use_graph=True)
    marg, mode, esc = pa.pa_uneven_run(h, len(blocks), info=True)
    torch.cuda.synchronize()
    assert any(c[3] > 1 for c in pa.pa_uneven_classes(h))  # at least one three-level class
    check_blocks(sizes, data, blocks, nrows=65536, h=h)
    assert esc == 0 and max(marg) < 0.125  # transform length 2^24: well inside the 0.25 guard
    pa.pa_uneven_destroy(h)


def test_uneven_update_and_rerun_graph():
    sizes = SMALL[:7]
    d1 = inputs.uneven_block_inputs(sizes, base_seed=1)
    d2 = inputs.uneven_block_inputs(sizes, base_seed=2)
    b1 = device_blocks(sizes, d1)
    b2 = device_blocks(sizes, d2)
    h = pa.pa_uneven_create(b1, pa.PA_FP32_GUARD, use_graph=True)
    pa.pa_uneven_run(h, len(b1))
    torch.cuda.synchronize()
    check_blocks(sizes, d1, b1)
    pa.pa_uneven_update(h, b2)
    pa.pa_uneven_run(h, len(b2))
    torch.cuda.synchronize()
    check_blocks(sizes, d2, b2)
    pa.pa_uneven_destroy(h)


def test_uneven_forced_escalation():
    sizes = SMALL[4:9]
    data = inputs.uneven_block_inputs(sizes, base_seed=8)
    blocks = device_blocks(sizes, data)
    h = pa.pa_uneven_create(blocks, pa.PA_FP32_GUARD, use_graph=True)
    pa.pa_uneven_set_guard(h, -1.0)
    marg, mode, esc = pa.pa_uneven_run(h, len(blocks), info=True)
    torch.cuda.synchronize()
    assert esc == len(sizes) and all(md == pa.PA_FP64 for md in mode)
    check_blocks(sizes, data, blocks)
    pa.pa_uneven_destroy(h)


def test_block_alone_equals_block_in_mix():
    sizes = SMALL
    data = inputs.uneven_block_inputs(sizes, base_seed=4)
    mix = device_blocks(sizes, data)
    h = pa.pa_uneven_create(mix, pa.PA_FP32_GUARD, use_graph=True)
    pa.pa_uneven_run(h, len(mix))
    torch.cuda.synchronize()
    for b in [0, 3, 7, 9]:
        alone = device_blocks([sizes[b]], [data[b]])
        pa.pa_hash_uneven(alone, pa.PA_FP32_GUARD)
        torch.cuda.synchronize()
        assert torch.equal(alone[0][4], mix[b][4])
    pa.pa_uneven_destroy(h)


def test_uneven_256_block_workload():
    """256 blocks, n log-uniform in [2^16, 2^24], m/n uniform in [0.05, 0.6], graph captured."""
    sizes = inputs.uneven_sizes(256, base_seed=0)
    data = inputs.uneven_block_inputs(sizes, base_seed=0)
    blocks = device_blocks(sizes, data)
    h = pa.pa_uneven_create(blocks, pa.PA_FP32_GUARD, use_graph=True)
    marg, mode, esc = pa.pa_uneven_run(h, len(blocks), info=True)
    torch.cuda.synchronize()
    assert esc == 0 and max(marg) < 0.2  # lengths up to 2^25 with the Eq. 5-10 split; guard is 0.25
    # every block with n <= 2^20 whole, the larger ones on rows covering every digit of their split
    check_blocks(sizes, data, blocks, full_limit=1 << 20, nrows=2048, h=h)
    pa.pa_uneven_destroy(h)

"""Reduced-precision storage study (paper Section 5: how much precision the FFT needs).

pa_plan_set_storage_bits rounds every value stored between passes to a narrower
significand (10 bits as in FP16, 7 as in BF16) while the butterflies stay FP32. The
rounding margin max|w - rint(w)| grows as the significand shrinks; with the guard on,
every key whose margin exceeds 0.25 is recomputed in FP64, so the output bits stay
exact whatever the storage width.
"""
import numpy as np
import pytest
import torch

import paper_1809_07592_gb300 as pa
from oracle import oracle
from paper_1809_07592_gb300 import inputs
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

BITS = [23, 16, 13, 10, 7]  # FP32 as stored now, then narrower significands (10: FP16's, 7: BF16's)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_07592_gb300 import build
    build.build()
    pa.lib()


def run(n, m, keys, seed, bits, guard):
    p = pa.Plan(n, m, pa.PA_FP32_GUARD)
    pa.pa_plan_set_storage_bits(p.handle, bits)
    pa.pa_plan_set_guard(p.handle, guard)
    p.set_seed(to_dev(seed)[0])
    out, (marg, mode, esc) = p.hash(to_dev(keys), info=True)
    torch.cuda.synchronize()
    res = to_host(out, (m + 63) // 64)
    p.close()
    return res, np.array(marg), np.array(mode), esc


@pytest.mark.parametrize("lg", [16, 18, 20])
def test_storage_width_margins_and_exact_bits(lg):
    n = 1 << lg
    m = n // 4
    seed = inputs.bernoulli_bits(lg, 1, n + m - 1)
    keys = inputs.batch_keys(n, 4, base_seed=lg)
    ref, *_ = run(n, m, keys, seed, 23, 0.25)
    for k in (0, 3):
        np.testing.assert_array_equal(ref[k], oracle.toeplitz_hash(n, m, seed, keys[k]), err_msg=f"key {k}")
    raw = {}
    for bits in BITS:
        # guard off: the margins of the reduced-width transform itself
        _, marg, mode, esc = run(n, m, keys, seed, bits, 1e9)
        assert esc == 0 and (mode == pa.PA_FP32_GUARD).all()
        raw[bits] = float(marg.max())
        # guard on: keys over 0.25 go to FP64, and every output bit equals the full-width result
        got, marg2, mode2, esc2 = run(n, m, keys, seed, bits, 0.25)
        np.testing.assert_array_equal(got, ref, err_msg=f"{bits} significand bits")
        assert esc2 == int((marg > 0.25).sum())
        assert all(md == (pa.PA_FP64 if mg > 0.25 else pa.PA_FP32_GUARD) for md, mg in zip(mode2, marg))
    assert raw[23] < 0.05
    # a narrower significand never gives a smaller rounding error than FP32 storage
    assert all(raw[b] >= raw[23] for b in BITS)
    # 7 significand bits (BF16's) leave no usable margin at these lengths
    assert raw[7] > 0.25

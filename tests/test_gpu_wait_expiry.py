"""The device-side wait limit: a staged last-pass launch whose copy wait runs out.

The staged last pass (pa_plan_set_staged; FP32 plans with a first pass of at most 256
values) copies its input tiles with tiled asynchronous copies and waits for each with a
time limit; a wait that runs out
sets the plan's device error word and the kernel returns, so the GPU stays usable. pa_plan_expire_waits arms a test hook that makes the next launch issue no copy
and wait on a barrier phase nothing completes (10 us), i.e. the wait certainly runs out
with nothing in flight. The synchronising call must report PA_ETIMEOUT and clear the
word; the next batch on the same plan must be bit-exact.
"""
import numpy as np
import pytest
import torch

import paper_1809_07592_gb300 as pa
from oracle import oracle
from paper_1809_07592_gb300 import inputs
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

# n + m - 1 = 999,999: transform length 2^20; split 256 x 4096 runs the staged last pass
N, M, SPLIT = 800_000, 200_000, (256, 4096, 1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_07592_gb300 import build
    build.build()
    pa.lib()


def _plan(seed):
    plan = pa.Plan(N, M, pa.PA_FP32_GUARD, split=SPLIT)
    assert tuple(plan.shape()) == (1 << 20,) + SPLIT
    pa.pa_plan_set_staged(plan.handle, True)
    plan.set_seed(to_dev(seed)[0])
    return plan


@pytest.mark.parametrize("issue", ["sync", "async"])
def test_expired_wait_reports_timeout_then_plan_recovers(issue):
    seed = inputs.bernoulli_bits(61, 1, N + M - 1)
    keys = inputs.batch_keys(N, 4, base_seed=61)
    kd = to_dev(keys)
    plan = _plan(seed)
    ow = (M + 63) // 64
    out = torch.zeros((4, ow + (ow & 1)), dtype=torch.int64, device="cuda")
    pa.pa_plan_expire_waits(plan.handle, 1)
    with pytest.raises(pa.PAError) as e:
        if issue == "sync":
            pa.pa_hash_batch(plan.handle, kd, 4, kd.shape[1], out, out.shape[1])
        else:
            pa.pa_hash_batch_async(plan.handle, kd, 4, kd.shape[1], out, out.shape[1])
            pa.pa_batch_finish(plan.handle, 4)
    assert e.value.code == pa.PA_ETIMEOUT
    torch.cuda.synchronize()  # the context is still usable
    # the hook disarmed itself and the error word was cleared: the next batch is exact
    marg, mode, esc = pa.pa_hash_batch(plan.handle, kd, 4, kd.shape[1], out, out.shape[1], info=True)
    torch.cuda.synchronize()
    got = to_host(out, ow)
    for k in range(4):
        np.testing.assert_array_equal(got[k], oracle.toeplitz_hash(N, M, seed, keys[k]), err_msg=f"key {k}")
    assert esc == 0 and max(marg) < 0.05
    plan.close()


def test_expire_hook_rejected_without_staged_pass():
    for dtype, staged in ((pa.PA_FP64, True), (pa.PA_FP32_GUARD, False)):  # FP64 plans never stage
        plan = pa.Plan(N, M, dtype)
        pa.pa_plan_set_staged(plan.handle, staged)
        with pytest.raises(pa.PAError) as e:
            pa.pa_plan_expire_waits(plan.handle, 1)
        assert e.value.code == pa.PA_EUNSUPPORTED
        plan.close()

"""One hash batch for profilers: ``python -m paper_1809_07592_gb300.profile_case``.

Sets up one plan (split autotuning, seed spectrum, one warm-up batch), then hashes
one batch of keys between cudaProfilerStart and cudaProfilerStop, so a profiler
run with ``--profile-from-start off`` sees exactly one launch of each pass kernel.
``--split L1,L2,L3`` fixes the pass split instead of autotuning it. ``--uneven B``
profiles an uneven batch instead: the B blocks of ``inputs.uneven_sizes(B)`` with
their own keys and seeds (streams 2b+2, 2b+3), replayed from their CUDA graph (one
warm-up run, then one run between the profiler calls). Inputs are the seeded
synthetic keys of ``inputs.py``; the CUDA path runs through the C ABI as in any
other call.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--m", type=int, default=1 << 18)
    ap.add_argument("--keys", type=int, default=32)
    ap.add_argument("--dtype", default="fp32_guard", choices=["fp32_guard", "fp64", "ntt64"])
    ap.add_argument("--split", default=None, help="L1,L2,L3 (one of pa_plan_splits); default: autotuned")
    ap.add_argument("--uneven", type=int, default=0, help="profile an uneven batch of this many blocks instead")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import paper_1809_07592_gb300 as pa
    from paper_1809_07592_gb300 import inputs

    torch.cuda.set_device(0)
    if a.uneven:
        return uneven(pa, inputs, torch, a.uneven)
    seed = inputs.bernoulli_bits(0, inputs.STREAM_SEED, a.n + a.m - 1)
    keys = inputs.batch_keys(a.n, a.keys, 0)
    kw = keys.shape[1] + (keys.shape[1] & 1)
    kb = np.zeros((a.keys, kw), np.uint64)
    kb[:, : keys.shape[1]] = keys
    sw = np.zeros(seed.size + (seed.size & 1), np.uint64)
    sw[: seed.size] = seed
    split = tuple(int(x) for x in a.split.split(",")) if a.split else None
    plan = pa.Plan(a.n, a.m, a.dtype, split=split)
    plan.set_seed(torch.from_numpy(sw.view(np.int64)).cuda())
    dk = torch.from_numpy(kb.view(np.int64)).cuda()
    plan.hash(dk)  # warm-up
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    plan.hash(dk)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("ok", plan.shape())
    plan.close()
    return 0


def uneven(pa, inputs, torch, nblocks: int) -> int:
    def words(bits):
        w = np.zeros(bits.size + (bits.size & 1), np.uint64)
        w[: bits.size] = bits
        return torch.from_numpy(w.view(np.int64)).cuda()

    sizes = inputs.uneven_sizes(nblocks, base_seed=0)
    blocks = []
    for b, (n, m) in enumerate(sizes):
        ow = (m + 63) // 64
        blocks.append((n, m, words(inputs.bernoulli_bits(0, 2 * b + 2, n)),
                       words(inputs.bernoulli_bits(0, 2 * b + 3, n + m - 1)),
                       torch.empty(ow + (ow & 1), dtype=torch.int64, device="cuda")))
    h = pa.pa_uneven_create(blocks, pa.PA_FP32_GUARD, use_graph=True)
    pa.pa_uneven_run(h, len(blocks))  # warm-up
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    pa.pa_uneven_run(h, len(blocks))
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("ok", "classes (L, split..., blocks):", pa.pa_uneven_classes(h))
    print("sum n", sum(n for n, _ in sizes), "sum m", sum(m for _, m in sizes))
    pa.pa_uneven_destroy(h)
    return 0


if __name__ == "__main__":
    sys.exit(main())

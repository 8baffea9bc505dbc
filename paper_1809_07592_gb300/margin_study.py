"""Rounding margins of the FP32 and FP64 transforms across key lengths.

``python -m paper_1809_07592_gb300.margin_study [--keys K] [--max-lg 27]`` hashes K random
keys (shared seed) per size n = 2^16 .. 2^max-lg, m = n/4, in FP32_GUARD and FP64 with the
guard disabled (threshold 1.0, so no key is recomputed), and prints the largest and the mean
rounding margin max_i |w_i - rint(w_i)| per mode. The guard escalates a key when its margin
exceeds 0.25 (paper Section 5's precision question; the hash itself is exact whenever the
true error stays below 0.5). Inputs are the seeded synthetic keys of ``inputs.py``.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--keys", type=int, default=16)
    ap.add_argument("--min-lg", type=int, default=16)
    ap.add_argument("--max-lg", type=int, default=27)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import paper_1809_07592_gb300 as pa
    from paper_1809_07592_gb300 import inputs

    torch.cuda.set_device(0)
    for lg in range(a.min_lg, a.max_lg + 1):
        n = 1 << lg
        m = n // 4
        nk = a.keys if lg <= 24 else max(2, a.keys // 8)
        seed = inputs.bernoulli_bits(lg, 1, n + m - 1)
        keys = inputs.batch_keys(n, nk, base_seed=lg)
        kw = keys.shape[1] + (keys.shape[1] & 1)
        kb = np.zeros((nk, kw), np.uint64)
        kb[:, : keys.shape[1]] = keys
        sw = np.zeros(seed.size + (seed.size & 1), np.uint64)
        sw[: seed.size] = seed
        dk = torch.from_numpy(kb.view(np.int64)).cuda()
        row = {"n": n, "m": m, "keys": nk}
        for name, dt in (("fp32", pa.PA_FP32_GUARD), ("fp64", pa.PA_FP64)):
            plan = pa.Plan(n, m, dt)
            pa.pa_plan_set_guard(plan.handle, 1.0)
            plan.set_seed(torch.from_numpy(sw.view(np.int64)).cuda())
            _, (marg, mode, esc) = plan.hash(dk, info=True)
            row[name] = {"max_margin": float(max(marg)), "mean_margin": float(np.mean(marg)), "L": plan.shape()[0]}
            plan.close()
        print(json.dumps(row), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

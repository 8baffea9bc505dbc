"""Shared helpers for the GPU tests: device tensors of packed bits."""
import numpy as np
import torch

from paper_1809_07592_gb300 import inputs


def to_dev(words: np.ndarray, stride: int | None = None) -> torch.Tensor:
    """(nkeys, nwords) or (nwords,) uint64 -> int64 CUDA tensor, rows padded to ``stride`` words."""
    a = np.atleast_2d(np.ascontiguousarray(words, dtype=np.uint64))
    if stride is None:
        stride = a.shape[1] + (a.shape[1] & 1)
    buf = np.zeros((a.shape[0], stride), dtype=np.uint64)
    buf[:, : a.shape[1]] = a
    return torch.from_numpy(buf.view(np.int64)).cuda()


def to_host(t: torch.Tensor, nwords: int) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)[:, :nwords]


def unpack_rows(words: np.ndarray, nbits: int) -> np.ndarray:
    return np.stack([inputs.unpack(w, nbits) for w in np.atleast_2d(words)])


def sample_rows(m: int, k: int, seed: int = 0) -> np.ndarray:
    """Rows to spot-check: both ends, word boundaries and random interior rows."""
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 31, 32, 63, 64, 65, m // 2, m - 65, m - 64, m - 2, m - 1]
    rows = np.unique(np.concatenate([[r for r in fixed if 0 <= r < m], rng.integers(0, m, k)]))
    return rows.astype(np.uint64)


def cover_rows(m: int, shape, count: int = 65536, tail: int = 2048) -> np.ndarray:
    """Rows for a full-size check where the oracle cannot afford all m rows.

    ``shape`` is a plan's (L, L1, L2, L3) as pa_plan_shape reports it. Output row t sits at
    t = a1*S + a2*L3 + a3 (three passes, S = L2*L3) or t = a1*S + a2 (two passes, S = L2):
    a1 is the row's element in the strided first/last pass, the other digits its column.
    The rows below take every value of every column digit (every residue of t modulo the
    innermost length and, for three passes, every value of the middle pass's element) and
    every first-pass element that holds only outputs, plus the first and last ``tail`` rows
    (the partial last first-pass element and the word boundaries at both ends).
    """
    L, L1, L2, L3 = (int(x) for x in shape)
    inner = [L3, L2] if L3 > 1 else [L2]  # column digits, innermost first
    S = int(np.prod(inner))
    A1 = m // S  # first-pass elements all of whose rows are outputs
    if A1 == 0:
        rows = np.arange(min(m, count), dtype=np.int64)
    else:
        k = np.arange(max(count, max(inner)), dtype=np.int64)
        rows = (k * 2654435761 % A1) * S  # 2654435761 is prime: every a1 < A1 occurs
        place = 1
        for j, ln in enumerate(inner):
            # innermost digit: k mod ln; the middle strided digit (a power of two): an odd multiplier
            c = 1 if j == 0 else 40503
            rows += ((k * c) % ln) * place
            place *= ln
    ends = np.concatenate([np.arange(min(tail, m)), np.arange(max(0, m - tail), m)])
    rows = np.unique(np.concatenate([rows, ends]))
    if rows.size < min(count, m):  # top up with seeded random rows
        extra = np.random.default_rng(m).integers(0, m, 2 * (count - rows.size) + 64)
        rows = np.unique(np.concatenate([rows, extra]))
    return rows.astype(np.uint64)

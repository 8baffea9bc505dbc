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

"""Independent checks that pin the oracle (and, through it, the CUDA path).

Nothing here calls the oracle or the CUDA library; these are separate routes
to the same numbers, written from the paper's definitions:

* ``dense_toeplitz`` builds T from its first row and first column, the way
  Section 2.2 describes a Toeplitz matrix ("constructed by its first column and
  first row"), and ``brute_hash`` multiplies it out over GF(2).
* ``circulant_fp64`` embeds T in a circulant of length L >= n+m-1 and
  evaluates the product with real FFTs in double precision (Eq. 4's
  convolution theorem), rounding the exact integer counts.
* ``paper_orientation_hash`` evaluates the consistent reading of the
  matrix layout printed in Eq. 2 (entry (i, j) of the Toeplitz block is
  V_{r-1-i+j}), used to pin the orientation reading.
"""
from __future__ import annotations

import numpy as np


def bits_of(words: np.ndarray, nbits: int) -> np.ndarray:
    b = np.unpackbits(np.ascontiguousarray(words, dtype="<u8").view(np.uint8), bitorder="little")
    return b[:nbits].astype(np.int64)


def words_of(bits) -> np.ndarray:
    bits = np.asarray(bits, dtype=np.uint8) & 1
    nw = (bits.size + 63) // 64
    pad = np.zeros(nw * 64, dtype=np.uint8)
    pad[: bits.size] = bits
    return np.packbits(pad, bitorder="little").view("<u8").astype(np.uint64)


def first_row_col(n: int, m: int, s: np.ndarray):
    """First row and first column of the m x n Toeplitz matrix of seed s.

    Row 0 is s[n-1], s[n-2], ..., s[0]; column 0 is s[n-1], s[n], ..., s[n+m-2].
    """
    row = np.array([s[n - 1 - j] for j in range(n)], dtype=np.int64)
    col = np.array([s[n - 1 + i] for i in range(m)], dtype=np.int64)
    return row, col


def dense_toeplitz(n: int, m: int, s: np.ndarray) -> np.ndarray:
    """T[i][j] = col[i-j] below the diagonal, row[j-i] on and above it."""
    row, col = first_row_col(n, m, s)
    T = np.zeros((m, n), dtype=np.int64)
    for i in range(m):
        for j in range(n):
            T[i, j] = col[i - j] if i >= j else row[j - i]
    return T


def brute_hash(n: int, m: int, s_bits: np.ndarray, x_bits: np.ndarray) -> np.ndarray:
    T = dense_toeplitz(n, m, s_bits)
    return (T @ np.asarray(x_bits, dtype=np.int64)) % 2


def circulant_fp64(n: int, m: int, s_bits: np.ndarray, x_bits: np.ndarray, L: int | None = None):
    """(y bits, max distance of the FP64 counts from the nearest integer).

    Linear convolution c = s * x through a cyclic convolution of length
    L >= n+m-1 (no wrap-around reaches the kept window), y_i = c[i+n-1] mod 2.
    """
    need = n + m - 1
    if L is None:
        L = 1 << int(np.ceil(np.log2(max(need, 2))))
    assert L >= need
    xs = np.zeros(L)
    xs[:n] = x_bits
    ss = np.zeros(L)
    ss[:need] = s_bits[:need]
    c = np.fft.irfft(np.fft.rfft(xs) * np.fft.rfft(ss), L)[n - 1:n - 1 + m]
    r = np.rint(c)
    return (r.astype(np.int64) & 1), float(np.max(np.abs(c - r)) if m else 0.0)


def paper_orientation_hash(n: int, m: int, v_bits: np.ndarray, x_bits: np.ndarray) -> np.ndarray:
    """Toeplitz product in the orientation printed in Eq. 2: entry (i, j) = V_{m-1-i+j}.

    Here V has n+m-1 bits (the standard Toeplitz matrix of Section 2.2 laid out
    as the block of Eq. 2). Row 0 runs V_{m-1}, V_m, ...; the last row starts at V_0.
    """
    y = np.zeros(m, dtype=np.int64)
    for i in range(m):
        acc = 0
        for j in range(n):
            acc ^= int(v_bits[m - 1 - i + j]) & int(x_bits[j])
        y[i] = acc
    return y


def dense_modified(n: int, m: int, s: np.ndarray) -> np.ndarray:
    """The modified Toeplitz matrix of Section 2.2 (Eq. 2): [I_m | T'] with T' the m x (n-m)
    Toeplitz matrix of the (n-1)-bit seed s (built by dense_toeplitz from first row and column)."""
    S = np.zeros((m, n), dtype=np.int64)
    S[:, :m] = np.eye(m, dtype=np.int64)
    S[:, m:] = dense_toeplitz(n - m, m, s)
    return S


def paper_modified_hash(n: int, m: int, v_bits: np.ndarray, x_bits: np.ndarray) -> np.ndarray:
    """Eq. 2-3 in the layout the paper prints: identity on the first r = m columns, then the block
    V with entry (i, j) = V_{r-1-i+j}, j < n-r (V has n-1 bits); y = X_r + V X_(n-r)."""
    r = m
    y = np.zeros(m, dtype=np.int64)
    for i in range(m):
        acc = int(x_bits[i])
        for j in range(n - r):
            acc ^= int(v_bits[r - 1 - i + j]) & int(x_bits[r + j])
        y[i] = acc
    return y

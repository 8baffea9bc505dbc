"""CPU oracle for the Toeplitz hash y = T x mod 2 (ctypes binding of pa_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers. The CUDA
product path never imports this module and shares no code with it.

Definition followed (paper Section 2.2, Eq. 3-4): T is the m x n binary
Toeplitz matrix T[i][j] = s[i - j + n - 1] built from an (n+m-1)-bit seed s,
and the final key is y_i = XOR_j T[i][j] AND x_j. The C code evaluates that
definition directly (bit-parallel AND + popcount parity, O(n m)).

The modified Toeplitz hash of Section 2.2 (Eq. 2-3) is the identity block
next to a Toeplitz block: y = x_[0,m) XOR T' x_[m,n), T' the m x (n-m)
Toeplitz matrix of an (n-1)-bit seed. ``modified_hash`` evaluates Eq. 3's two
terms as written: the first m key bits, XOR the Toeplitz product (above) of
the remaining n-m key bits.

Pins (``tests/test_oracle_pins.py``): dense brute force for n <= 64 and every
key for tiny n, GF(2) linearity in key and seed, Toeplitz shift structure,
special cases (unit key, all-ones seed, single-one seed, m = 1), hand-worked
golden fixtures, and agreement with an independent FP64 circulant-embedding
convolution (Eq. 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libpa_oracle.so")
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile pa_oracle.c with the system C compiler (portable C11, -O2)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.pa_oracle_hash.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, _u64p, ctypes.c_int]
        lib.pa_oracle_hash.restype = ctypes.c_int
        lib.pa_oracle_hash_rows.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, ctypes.c_uint64,
                                            ctypes.c_uint64, _u64p, ctypes.c_int]
        lib.pa_oracle_hash_rows.restype = ctypes.c_int
        lib.pa_oracle_row.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, ctypes.c_uint64]
        lib.pa_oracle_row.restype = ctypes.c_int
        lib.pa_oracle_rows.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, _u64p, ctypes.c_uint64,
                                       _u8p, ctypes.c_int]
        lib.pa_oracle_rows.restype = ctypes.c_int
        _lib = lib
    return _lib


def _words(a, nbits: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    need = (nbits + 63) // 64
    if a.size < need:
        raise ValueError(f"bit-vector has {a.size} words, needs {need}")
    return a


def default_threads() -> int:
    return os.cpu_count() or 1


def toeplitz_hash(n: int, m: int, seed, key, threads: int | None = None) -> np.ndarray:
    """All m output bits, packed into ceil(m/64) uint64 words (tail zero)."""
    seed = _words(seed, n + m - 1)
    key = _words(key, n)
    out = np.zeros((m + 63) // 64, dtype=np.uint64)
    rc = _load().pa_oracle_hash(n, m, seed.ctypes.data_as(_u64p), key.ctypes.data_as(_u64p),
                                out.ctypes.data_as(_u64p), threads or default_threads())
    if rc != 0:
        raise ValueError(f"pa_oracle_hash rc={rc} (n={n}, m={m})")
    return out


def toeplitz_rows(n: int, m: int, seed, key, rows, threads: int | None = None) -> np.ndarray:
    """Selected output bits y_i for i in ``rows`` (uint8 array, one bit each)."""
    seed = _words(seed, n + m - 1)
    key = _words(key, n)
    rows = np.ascontiguousarray(rows, dtype=np.uint64)
    bits = np.zeros(rows.size, dtype=np.uint8)
    rc = _load().pa_oracle_rows(n, m, seed.ctypes.data_as(_u64p), key.ctypes.data_as(_u64p),
                                rows.ctypes.data_as(_u64p), rows.size, bits.ctypes.data_as(_u8p),
                                threads or default_threads())
    if rc != 0:
        raise ValueError(f"pa_oracle_rows rc={rc}")
    return bits


def toeplitz_row_range(n: int, m: int, seed, key, row0: int, row1: int, threads: int | None = None) -> np.ndarray:
    """Rows [row0, row1) into a zeroed ceil(m/64)-word buffer (other bits zero)."""
    seed = _words(seed, n + m - 1)
    key = _words(key, n)
    out = np.zeros((m + 63) // 64, dtype=np.uint64)
    rc = _load().pa_oracle_hash_rows(n, m, seed.ctypes.data_as(_u64p), key.ctypes.data_as(_u64p), row0, row1,
                                     out.ctypes.data_as(_u64p), threads or default_threads())
    if rc != 0:
        raise ValueError(f"pa_oracle_hash_rows rc={rc}")
    return out


def key_bits_from(key, nbits: int, start: int) -> np.ndarray:
    """Bits [start, nbits) of a packed bit-vector, repacked from bit 0 (tail zero)."""
    b = np.unpackbits(np.ascontiguousarray(key, dtype="<u8").view(np.uint8), bitorder="little")[start:nbits]
    nw = (b.size + 63) // 64
    pad = np.zeros(nw * 64, dtype=np.uint8)
    pad[: b.size] = b
    return np.packbits(pad, bitorder="little").view("<u8").astype(np.uint64)


def modified_hash(n: int, m: int, seed, key, threads: int | None = None) -> np.ndarray:
    """Eq. 3: y = X_r + V X_(n-r) with r = m, V the m x (n-m) Toeplitz block of the (n-1)-bit seed
    (entry (i, j) = seed[i - j + n - m - 1], the orientation of toeplitz_hash). 1 <= m < n."""
    if not 1 <= m < n:
        raise ValueError("the modified Toeplitz hash needs 1 <= m < n")
    key = _words(key, n)
    tail = key_bits_from(key, n, m)                    # X_(n-r): key bits m .. n-1
    y = toeplitz_hash(n - m, m, seed, tail, threads)   # V X_(n-r)
    head = key_bits_from(key, m, 0)                    # X_r: key bits 0 .. m-1
    return y ^ head


def modified_rows(n: int, m: int, seed, key, rows, threads: int | None = None) -> np.ndarray:
    """Selected output bits of modified_hash (uint8 array, one bit each)."""
    key = _words(key, n)
    tail = key_bits_from(key, n, m)
    y = toeplitz_rows(n - m, m, seed, tail, rows, threads)
    rows = np.asarray(rows, dtype=np.int64)
    head = np.unpackbits(np.ascontiguousarray(key, dtype="<u8").view(np.uint8), bitorder="little")[rows]
    return (y ^ head).astype(np.uint8)

"""Seeded synthetic inputs: packed Bernoulli(0.5) bit-vectors.

This module holds no arithmetic of the hashing method. It only draws the
keys and Toeplitz seeds that both the CUDA path and the CPU oracle consume.
Reconciled QKD keys are modelled as i.i.d. Bernoulli(0.5) bits (the paper's
input X_n of Section 2.3 and the n+r-1 random bits of the Toeplitz
description of Section 2.2).

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; constants as in S. Vigna's
public-domain reference). It is counter based: word ``w`` of a stream is
``mix(state0 + (w + 1) * GAMMA)``, so any slice can be drawn independently.

Stream convention: ``state0 = mix(base_seed ^ (stream_id * GAMMA))``.
Stream 0 is the key and stream 1 the seed of a single block; batched keys use
streams 2, 3, ...; block ``b`` of an uneven batch uses streams 2b+2 (key) and
2b+3 (seed).

Packed layout: bit ``j`` of a bit-vector lives in 64-bit word ``j // 64`` at
bit position ``j % 64`` (LSB first); bits at or past the vector's length in
the last word are zero.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_KEY = 0
STREAM_SEED = 1


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (variant 13 of Stafford's mixers)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_state(base_seed: int, stream_id: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(base_seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream_id) * GAMMA)
    return _mix(np.array([s], dtype=np.uint64))[0]


def words(base_seed: int, stream_id: int, nwords: int, offset: int = 0) -> np.ndarray:
    """``nwords`` raw 64-bit words of one stream, starting at word ``offset``."""
    s0 = stream_state(base_seed, stream_id)
    idx = np.arange(offset + 1, offset + nwords + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(s0 + idx * GAMMA)


def nwords_for(nbits: int) -> int:
    return (nbits + 63) // 64


def mask_tail(w: np.ndarray, nbits: int) -> np.ndarray:
    """Zero the bits at positions >= nbits (in place on a copy)."""
    w = np.array(w, dtype=np.uint64, copy=True)
    nw = nwords_for(nbits)
    w[nw:] = 0
    r = nbits % 64
    if r and nw:
        w[nw - 1] &= np.uint64((1 << r) - 1)
    return w


def bernoulli_bits(base_seed: int, stream_id: int, nbits: int) -> np.ndarray:
    """Packed i.i.d. Bernoulli(0.5) bit-vector of ``nbits`` bits."""
    return mask_tail(words(base_seed, stream_id, nwords_for(nbits)), nbits)


def block_inputs(n: int, m: int, base_seed: int = 0, key_stream: int = STREAM_KEY,
                 seed_stream: int = STREAM_SEED):
    """(key, seed) packed words for one block: n key bits, n+m-1 seed bits."""
    return (bernoulli_bits(base_seed, key_stream, n),
            bernoulli_bits(base_seed, seed_stream, n + m - 1))


def batch_keys(n: int, nkeys: int, base_seed: int = 0, first_stream: int = 2) -> np.ndarray:
    """(nkeys, ceil(n/64)) packed keys, key k drawn from stream first_stream+k."""
    nw = nwords_for(n)
    out = np.empty((nkeys, nw), dtype=np.uint64)
    for k in range(nkeys):
        out[k] = bernoulli_bits(base_seed, first_stream + k, n)
    return out


def unpack(words_: np.ndarray, nbits: int) -> np.ndarray:
    """Packed words -> uint8 array of nbits bits (LSB first)."""
    b = np.unpackbits(np.ascontiguousarray(words_, dtype="<u8").view(np.uint8), bitorder="little")
    return b[:nbits].copy()


def pack(bits: np.ndarray) -> np.ndarray:
    """uint8/bool bit array -> packed uint64 words (tail zero)."""
    bits = np.asarray(bits, dtype=np.uint8) & 1
    nb = bits.size
    nw = nwords_for(nb)
    padded = np.zeros(nw * 64, dtype=np.uint8)
    padded[:nb] = bits
    return np.packbits(padded, bitorder="little").view("<u8").astype(np.uint64)


def uniform01(base_seed: int, stream_id: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from the top 53 bits of a stream."""
    w = words(base_seed, stream_id, count)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


STREAM_UNEVEN_N = 1_000_001
STREAM_UNEVEN_M = 1_000_002


def uneven_sizes(nblocks: int, base_seed: int = 0, lg_lo: float = 16.0, lg_hi: float = 24.0,
                 ratio_lo: float = 0.05, ratio_hi: float = 0.6):
    """(n, m) for an uneven batch: n = floor(2^u), u ~ U[lg_lo, lg_hi]; m = floor(r n), r ~ U[ratio_lo, ratio_hi], m >= 1."""
    u = uniform01(base_seed, STREAM_UNEVEN_N, nblocks)
    r = uniform01(base_seed, STREAM_UNEVEN_M, nblocks)
    ns = np.floor(np.exp2(lg_lo + (lg_hi - lg_lo) * u)).astype(np.int64)
    ms = np.maximum(1, np.floor((ratio_lo + (ratio_hi - ratio_lo) * r) * ns)).astype(np.int64)
    ms = np.minimum(ms, ns)
    return [(int(n), int(m)) for n, m in zip(ns, ms)]


def uneven_block_inputs(sizes, base_seed: int = 0):
    """Keys (stream 2b+2) and seeds (stream 2b+3) for block b of an uneven batch."""
    return [(bernoulli_bits(base_seed, 2 * b + 2, n), bernoulli_bits(base_seed, 2 * b + 3, n + m - 1))
            for b, (n, m) in enumerate(sizes)]


STREAM_SERVE_N = 1_000_003
STREAM_SERVE_M = 1_000_004
STREAM_SERVE_T = 1_000_005
SERVE_N_CHOICES = (1 << 18, 1_000_000, 1 << 22, 1 << 24)
SERVE_N_WEIGHTS = (0.4, 0.3, 0.2, 0.1)


def serving_requests(count: int, rate_per_s: float, base_seed: int = 0, ratio_lo: float = 0.1,
                     ratio_hi: float = 0.5):
    """Arrival times (s, Poisson process of the given rate) and (n, m) for a serving run.

    n is drawn from SERVE_N_CHOICES with SERVE_N_WEIGHTS, m = floor(U[ratio_lo, ratio_hi] * n).
    """
    u_n = uniform01(base_seed, STREAM_SERVE_N, count)
    u_m = uniform01(base_seed, STREAM_SERVE_M, count)
    u_t = uniform01(base_seed, STREAM_SERVE_T, count)
    cum = np.cumsum(SERVE_N_WEIGHTS)
    idx = np.searchsorted(cum, u_n * cum[-1], side="right")
    ns = np.array(SERVE_N_CHOICES, dtype=np.int64)[np.minimum(idx, len(SERVE_N_CHOICES) - 1)]
    ms = np.maximum(1, np.floor((ratio_lo + (ratio_hi - ratio_lo) * u_m) * ns)).astype(np.int64)
    gaps = -np.log1p(-u_t) / rate_per_s  # exponential inter-arrival times
    return np.cumsum(gaps), [(int(n), int(m)) for n, m in zip(ns, ms)]

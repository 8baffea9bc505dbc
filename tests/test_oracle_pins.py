"""Pins for the CPU oracle (no GPU needed).

Each test ties the oracle to something other than itself: hand-worked
examples, a dense matrix built from the first row and column, GF(2)
linearity, the diagonal-constant (shift) structure, closed-form special
cases, the FP64 convolution-theorem route of Eq. 4 and the Eq. 2 orientation.
A final test plants mistakes in a copy of the oracle and checks that these
pins catch every one.
"""
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import oracle
from paper_1809_07592_gb300 import inputs
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toeplitz_worked_examples.txt")


def rand_bits(rng, nbits):
    return rng.integers(0, 2, nbits).astype(np.int64)


def ohash(n, m, s_bits, x_bits, threads=2):
    return pins.bits_of(oracle.toeplitz_hash(n, m, pins.words_of(s_bits), pins.words_of(x_bits), threads), m)


def parse_golden():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, rows, y = [p.strip() for p in line.split("|")]
        n, m, s, x = head.split()
        n, m = int(n), int(m)
        cases.append((n, m, np.array([int(c) for c in s]), np.array([int(c) for c in x]),
                      [np.array([int(c) for c in r]) for r in rows.split("/")], np.array([int(c) for c in y])))
    return cases


@pytest.mark.parametrize("case", parse_golden(), ids=lambda c: f"n{c[0]}m{c[1]}")
def test_golden_worked_examples(case):
    n, m, s, x, rows, y = case
    assert s.size == n + m - 1 and x.size == n and y.size == m
    T = pins.dense_toeplitz(n, m, s)
    for i in range(m):
        np.testing.assert_array_equal(T[i], rows[i])
    np.testing.assert_array_equal(ohash(n, m, s, x), y)


def test_dense_is_diagonal_constant():
    rng = np.random.default_rng(1)
    n, m = 13, 7
    s = rand_bits(rng, n + m - 1)
    T = pins.dense_toeplitz(n, m, s)
    for i in range(m - 1):
        for j in range(n - 1):
            assert T[i, j] == T[i + 1, j + 1]
    # every seed bit appears on exactly one diagonal
    diag_vals = [T[max(0, d), max(0, -d)] for d in range(-(n - 1), m)]
    assert sorted(diag_vals) == sorted(s.tolist())


@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (5, 3), (17, 17), (63, 20), (64, 64), (65, 1), (64, 33)])
def test_brute_force_random(n, m):
    rng = np.random.default_rng(n * 1000 + m)
    for _ in range(6):
        s = rand_bits(rng, n + m - 1)
        x = rand_bits(rng, n)
        np.testing.assert_array_equal(ohash(n, m, s, x), pins.brute_hash(n, m, s, x))


@pytest.mark.parametrize("n,m", [(6, 3), (9, 9), (10, 4)])
def test_brute_force_every_key(n, m):
    rng = np.random.default_rng(7 + n)
    s = rand_bits(rng, n + m - 1)
    T = pins.dense_toeplitz(n, m, s)
    sw = pins.words_of(s)
    for v in range(1 << n):
        x = np.array([(v >> j) & 1 for j in range(n)])
        got = pins.bits_of(oracle.toeplitz_hash(n, m, sw, pins.words_of(x), 1), m)
        np.testing.assert_array_equal(got, (T @ x) % 2)


def test_linearity_in_key_and_seed():
    rng = np.random.default_rng(3)
    for n, m in [(200, 50), (1000, 999), (4096, 1024), (777, 130)]:
        s1, s2 = rand_bits(rng, n + m - 1), rand_bits(rng, n + m - 1)
        x1, x2 = rand_bits(rng, n), rand_bits(rng, n)
        np.testing.assert_array_equal(ohash(n, m, s1, x1 ^ x2), ohash(n, m, s1, x1) ^ ohash(n, m, s1, x2))
        np.testing.assert_array_equal(ohash(n, m, s1 ^ s2, x1), ohash(n, m, s1, x1) ^ ohash(n, m, s2, x1))
        assert not ohash(n, m, s1, np.zeros(n, dtype=np.int64)).any()
        assert not ohash(n, m, np.zeros(n + m - 1, dtype=np.int64), x1).any()


def test_shift_structure():
    rng = np.random.default_rng(4)
    for n, m in [(100, 40), (1000, 333), (130, 1)]:
        s = rand_bits(rng, n + m)  # seed of the (m+1)-row matrix
        x = rand_bits(rng, n)
        big = ohash(n, m + 1, s, x)
        np.testing.assert_array_equal(big[1:], ohash(n, m, s[1:], x))
        np.testing.assert_array_equal(big[:-1], ohash(n, m, s[:-1], x))


def test_special_cases():
    rng = np.random.default_rng(5)
    n, m = 300, 120
    s = rand_bits(rng, n + m - 1)
    x = rand_bits(rng, n)
    # unit key e_j picks column j: y_i = s[i - j + n - 1]
    for j in [0, 1, 150, n - 1]:
        e = np.zeros(n, dtype=np.int64)
        e[j] = 1
        np.testing.assert_array_equal(ohash(n, m, s, e), s[np.arange(m) - j + n - 1])
    # all-ones seed: every row sums the whole key
    np.testing.assert_array_equal(ohash(n, m, np.ones(n + m - 1, dtype=np.int64), x), np.full(m, x.sum() % 2))
    # all-ones key: y_i = parity of the seed window s[i .. i+n-1]
    exp = np.array([s[i:i + n].sum() % 2 for i in range(m)])
    np.testing.assert_array_equal(ohash(n, m, s, np.ones(n, dtype=np.int64)), exp)
    # single one in the seed at p: y_i = x[i + n - 1 - p] when in range
    for p in [0, 5, n - 1, n + m - 2]:
        sp = np.zeros(n + m - 1, dtype=np.int64)
        sp[p] = 1
        exp = np.array([x[i + n - 1 - p] if 0 <= i + n - 1 - p < n else 0 for i in range(m)])
        np.testing.assert_array_equal(ohash(n, m, sp, x), exp)
    # m = 1: a single inner product with the reversed first n seed bits
    np.testing.assert_array_equal(ohash(n, 1, s[:n], x), [int((s[:n][::-1] * x).sum() % 2)])


def test_paper_orientation_equivalence():
    """Eq. 2's layout (entry V_{r-1-i+j}) is the same map with the seed reversed."""
    rng = np.random.default_rng(6)
    for n, m in [(20, 7), (33, 33), (64, 5)]:
        s = rand_bits(rng, n + m - 1)
        x = rand_bits(rng, n)
        np.testing.assert_array_equal(ohash(n, m, s, x), pins.paper_orientation_hash(n, m, s[::-1].copy(), x))


@pytest.mark.parametrize("n,m", [(1, 1), (64, 64), (1000, 100), (4096, 4096), (10000, 2500), (65536, 6554),
                                 (131072, 32768)])
def test_circulant_fp64_agrees(n, m):
    """Eq. 4: the hash equals the rounded FFT convolution window, for every admissible L."""
    key, seed = inputs.block_inputs(n, m, base_seed=11)
    x = pins.bits_of(key, n)
    s = pins.bits_of(seed, n + m - 1)
    got = pins.bits_of(oracle.toeplitz_hash(n, m, seed, key), m)
    need = n + m - 1
    for L in sorted({need, need + 1, 1 << int(np.ceil(np.log2(max(need, 2)))), 2 * need + 3}):
        y, margin = pins.circulant_fp64(n, m, s, x, L)
        assert margin < 1e-3
        np.testing.assert_array_equal(got, y)


def test_packed_tails_ignored_and_zeroed():
    rng = np.random.default_rng(8)
    n, m = 100, 70
    s = rand_bits(rng, n + m - 1)
    x = rand_bits(rng, n)
    sw, xw = pins.words_of(s), pins.words_of(x)
    ref = oracle.toeplitz_hash(n, m, sw, xw)
    # garbage in the unused high bits of the last key / seed word must not matter
    xw2, sw2 = xw.copy(), sw.copy()
    xw2[-1] |= np.uint64(0xFFFFFFFFFFFFFFFF) << np.uint64(n % 64)
    sw2[-1] |= np.uint64(0xFFFFFFFFFFFFFFFF) << np.uint64((n + m - 1) % 64)
    got = oracle.toeplitz_hash(n, m, sw2, xw2)
    np.testing.assert_array_equal(ref, got)
    assert int(got[-1]) >> (m % 64) == 0


def test_row_helpers_match_full_hash():
    n, m = 5000, 3000
    key, seed = inputs.block_inputs(n, m, base_seed=2)
    full = pins.bits_of(oracle.toeplitz_hash(n, m, seed, key), m)
    rows = np.array([0, 1, 63, 64, 65, 1000, m - 2, m - 1], dtype=np.uint64)
    np.testing.assert_array_equal(oracle.toeplitz_rows(n, m, seed, key, rows), full[rows.astype(np.int64)])
    part = pins.bits_of(oracle.toeplitz_row_range(n, m, seed, key, 100, 700), m)
    np.testing.assert_array_equal(part[100:700], full[100:700])
    assert not part[:100].any() and not part[700:].any()


def test_generator_reference_values():
    """SplitMix64 published sequence for state 0 (Vigna's reference implementation)."""
    z = inputs._mix(np.array([1, 2, 3], dtype=np.uint64) * inputs.GAMMA)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    a = inputs.words(0, 5, 100)
    b = inputs.words(0, 5, 40, offset=60)
    np.testing.assert_array_equal(a[60:], b)
    k = inputs.bernoulli_bits(0, 0, 1000)
    assert int(k[-1]) >> (1000 % 64) == 0
    frac = pins.bits_of(inputs.bernoulli_bits(0, 1, 1 << 16), 1 << 16).mean()
    assert abs(frac - 0.5) < 0.01


MUTATIONS = {
    "row_off_by_one": ("i + 64 * w) & xr[w]", "i + 1 + 64 * w) & xr[w]"),
    "key_not_reversed": ("get_bit(key, n - 1 - j)", "get_bit(key, j)"),
    "dropped_last_word": ("for (uint64_t w = 0; w < nw; ++w) acc", "for (uint64_t w = 0; w + 1 < nw; ++w) acc"),
    "seed_window_short": ("uint64_t sbits = n + m - 1;", "uint64_t sbits = n + m - 2;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(name, tmp_path):
    """Plant a mistake in a copy of the oracle; brute force or Eq. 4 must reject it."""
    import ctypes
    src = open(os.path.join(os.path.dirname(oracle.__file__), "pa_oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, name
    mutated = src.replace(old, new)
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(mutated)
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-pthread", str(c), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.pa_oracle_hash.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u64p, u64p, u64p, ctypes.c_int]
    caught = False
    rng = np.random.default_rng(9)
    for n, m in [(5, 3), (64, 64), (130, 70), (1000, 500)]:
        s, x = rand_bits(rng, n + m - 1), rand_bits(rng, n)
        sw, xw = pins.words_of(s), pins.words_of(x)
        out = np.zeros((m + 63) // 64, dtype=np.uint64)
        lib.pa_oracle_hash(n, m, sw.ctypes.data_as(u64p), xw.ctypes.data_as(u64p), out.ctypes.data_as(u64p), 1)
        got = pins.bits_of(out, m)
        exp = pins.brute_hash(n, m, s, x) if n <= 130 else pins.circulant_fp64(n, m, s, x)[0]
        if not np.array_equal(got, exp):
            caught = True
            break
    assert caught, f"planted mistake {name} was not caught"


# ---- modified Toeplitz matrix (Section 2.2, Eq. 2-3) ---------------------------------------------
@pytest.mark.parametrize("n,m", [(2, 1), (5, 2), (17, 16), (33, 7), (64, 1), (64, 63), (65, 30), (130, 65)])
def test_modified_brute_force(n, m):
    """[I_m | T'] x mod 2 written out densely equals the oracle's Eq. 3 evaluation."""
    rng = np.random.default_rng(n * 1000 + m)
    s = rng.integers(0, 2, n - 1)
    x = rng.integers(0, 2, n)
    exp = (pins.dense_modified(n, m, s) @ x) % 2
    got = pins.bits_of(oracle.modified_hash(n, m, pins.words_of(s), pins.words_of(x)), m)
    np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("n,m", [(9, 4), (40, 13), (100, 99)])
def test_modified_paper_orientation(n, m):
    """The paper's printed layout (V_{r-1-i+j}) is the same hash with the seed reversed."""
    rng = np.random.default_rng(7 * n + m)
    s = rng.integers(0, 2, n - 1)
    x = rng.integers(0, 2, n)
    got = pins.bits_of(oracle.modified_hash(n, m, pins.words_of(s), pins.words_of(x)), m)
    np.testing.assert_array_equal(got, pins.paper_modified_hash(n, m, s[::-1].copy(), x))


def test_modified_special_cases():
    n, m = 300, 70
    rng = np.random.default_rng(3)
    s = rng.integers(0, 2, n - 1)
    x = rng.integers(0, 2, n)
    head = x[:m]
    # all-zero seed: the Toeplitz block vanishes, the final key is the first m key bits
    got = pins.bits_of(oracle.modified_hash(n, m, pins.words_of(np.zeros(n - 1, np.int64)), pins.words_of(x)), m)
    np.testing.assert_array_equal(got, head)
    # key zero past bit m: same
    x2 = x.copy()
    x2[m:] = 0
    got = pins.bits_of(oracle.modified_hash(n, m, pins.words_of(s), pins.words_of(x2)), m)
    np.testing.assert_array_equal(got, head)
    # key zero in its first m bits: the plain Toeplitz product of the remaining bits
    x3 = x.copy()
    x3[:m] = 0
    got = pins.bits_of(oracle.modified_hash(n, m, pins.words_of(s), pins.words_of(x3)), m)
    np.testing.assert_array_equal(got, pins.brute_hash(n - m, m, s, x3[m:]))
    # rows helper
    rows = np.array([0, 1, m // 2, m - 1], dtype=np.uint64)
    full = pins.bits_of(oracle.modified_hash(n, m, pins.words_of(s), pins.words_of(x)), m)
    np.testing.assert_array_equal(oracle.modified_rows(n, m, pins.words_of(s), pins.words_of(x), rows),
                                  full[rows.astype(np.int64)])
    with pytest.raises(ValueError):
        oracle.modified_hash(n, n, pins.words_of(s), pins.words_of(x))


def test_modified_linearity():
    n, m = 200, 61
    rng = np.random.default_rng(11)
    s = pins.words_of(rng.integers(0, 2, n - 1))
    a, b = pins.words_of(rng.integers(0, 2, n)), pins.words_of(rng.integers(0, 2, n))
    np.testing.assert_array_equal(oracle.modified_hash(n, m, s, a ^ b),
                                  oracle.modified_hash(n, m, s, a) ^ oracle.modified_hash(n, m, s, b))

"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

from paper_1809_07592_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pa_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_boundary():
    names = declared_functions()
    for required in ["pa_plan", "pa_plan_destroy", "pa_set_seed", "pa_hash_batch", "pa_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.pa_strerror.restype = ctypes.c_char_p
    assert lib.pa_strerror(0).startswith(b"PA_OK")
    assert lib.pa_strerror(-1).startswith(b"PA_EINVAL")


def test_no_library_fft_or_blas_linked():
    """The product links no cuFFT/cuBLAS: check the dynamic dependencies of libpa.so."""
    path = build.build()
    import subprocess
    deps = subprocess.run(["ldd", path], capture_output=True, text=True).stdout
    assert "cufft" not in deps and "cublas" not in deps


def test_split_listing_without_gpu():
    """pa_plan_splits is host-only: every listed split multiplies out to one length L >= n+m-1."""
    import paper_1809_07592_gb300 as pa
    build.build()
    for n, m, dtype in [(1 << 20, 1 << 18, pa.PA_FP32_GUARD), (1_000_000, 100_000, pa.PA_FP32_GUARD),
                        (1_000_000, 500_000, pa.PA_FP64), (1 << 20, 1 << 19, pa.PA_NTT64),
                        ((1 << 27), 1 << 24, pa.PA_FP32_GUARD), (5000, 1500, pa.PA_FP64)]:
        splits = pa.pa_plan_splits(n, m, dtype)
        assert splits, (n, m, dtype)
        lengths = {a * b * c for a, b, c in splits}
        assert len(lengths) == 1, splits
        L = lengths.pop()
        assert L >= n + m - 1 and L >= 4096
        assert len(set(splits)) == len(splits)
        if dtype == pa.PA_NTT64:
            assert L & (L - 1) == 0
    # the DV-QKD length 5 * 2^18 has a split for every level-1 pass 2^7 .. 2^10
    assert sorted(a for a, _, _ in pa.pa_plan_splits(1 << 20, 1 << 18, pa.PA_FP32_GUARD)) == [128, 256, 512, 1024]
    try:
        pa.pa_plan_splits(10, 11, pa.PA_FP64)
        raise AssertionError("m > n accepted")
    except pa.PAError as e:
        assert e.code == pa.PA_EINVAL


def test_security_parameter_helpers_without_gpu():
    """Eq. 1: r = n - t - s and the bound 2^-s / ln 2 (host-only entry points)."""
    import math
    import paper_1809_07592_gb300 as pa
    build.build()
    assert pa.pa_final_key_length(1_000_000, 400_000, 100) == 599_900
    assert pa.pa_final_key_length(10, 0, 9) == 1
    for n, t, s in [(10, 10, 0), (10, 3, 7), (10, 11, 0), (0, 0, 0)]:
        try:
            pa.pa_final_key_length(n, t, s)
            raise AssertionError((n, t, s))
        except pa.PAError as e:
            assert e.code == pa.PA_EINVAL
    assert math.isclose(pa.pa_leakage_bound(1000, 400, 500), 2.0 ** -100 / math.log(2), rel_tol=1e-12)
    assert math.isclose(pa.pa_leakage_bound(1000, 400, 600), 1 / math.log(2), rel_tol=1e-12)
    # the bound halves for every bit dropped from the final key
    assert math.isclose(pa.pa_leakage_bound(5000, 1000, 3900) / pa.pa_leakage_bound(5000, 1000, 3901), 0.5)


def test_plan_lengths_and_splits_sweep_without_gpu():
    """Plan invariants over 240 seeded (n, m), host only: every split multiplies out to the one
    transform length L >= n+m-1; L is smooth (odd part 1, 3, 5 or 9; a power of two for the exact
    mode); the strided passes are powers of two in [64, 1024] and the odd factor sits in the
    innermost pass; and from n+m-1 = 24576 on (the smallest smooth length a split can realise:
    a 64-point strided pass times a 3 * 128-point innermost row) L is the smallest length of the
    ladder {1, 3, 5, 9} * 2^k (odd factors with k >= 13) not below n+m-1."""
    import random

    import paper_1809_07592_gb300 as pa
    build.build()
    rng = random.Random(17)

    def odd(v):
        while v % 2 == 0:
            v //= 2
        return v

    def ladder_min(need, exact):
        best = 1 << 40
        for ro in ((1,) if exact else (1, 3, 5, 9)):
            k = 0 if ro == 1 else 13
            while (ro << k) < need:
                k += 1
            best = min(best, ro << k)
        return best

    for _ in range(80):
        n = max(1, int(2 ** rng.uniform(4, 27)))
        m = max(1, int(rng.uniform(0.01, 1.0) * n))
        need = n + m - 1
        for dtype in (pa.PA_FP32_GUARD, pa.PA_FP64, pa.PA_NTT64):
            splits = pa.pa_plan_splits(n, m, dtype)
            assert splits, (n, m, dtype)
            lengths = {a * b * c for a, b, c in splits}
            assert len(lengths) == 1, (n, m, dtype, splits)
            L = lengths.pop()
            exact = dtype == pa.PA_NTT64
            assert need <= L <= 1 << 28 and L >= 4096
            assert odd(L) in ((1,) if exact else (1, 3, 5, 9)), (n, m, dtype, L)
            for a, b, c in splits:
                inner = b if c == 1 else c
                strided = (a,) if c == 1 else (a, b)
                assert all(s & (s - 1) == 0 and 64 <= s <= 1024 for s in strided), splits
                assert odd(inner) == odd(L), splits
            if need >= 24576:
                assert L == ladder_min(need, exact), (n, m, dtype, L, ladder_min(need, exact))

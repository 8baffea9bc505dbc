"""Host-side arithmetic of bench.py (no GPU): the per-launch algorithmic bytes behind the
roofline's `achieved` figure, written out by hand for the DV-QKD batch n = 2^20, m = 2^18
(L = 5 * 2^18, 32 key pairs, 64 keys, FP32 slots of 8 bytes per complex value), and the
per-pass bytes and textbook work of the 2^27-bit long block."""
import math

import bench


def test_algorithmic_bytes_per_launch():
    n, m, L, pairs, nkeys = 1 << 20, 1 << 18, 1310720, 32, 64
    slot = 8 * L                        # one key pair's complex work slot
    keys = nkeys * (n // 64) * 8        # packed key words read
    outs = nkeys * (m // 64) * 8        # packed final-key words written
    ab = lambda k: bench.algorithmic_bytes(k, n, m, L, pairs, nkeys, 8)
    assert ab("fwd_keys") == pairs * slot + keys == 343_932_928        # write W, read the bits
    assert ab("middle_conv") == 2 * pairs * slot + slot == 681_574_400  # W in, W out, spectrum once
    assert ab("inv_bits") == pairs * slot + outs == 337_641_472        # read W, write the bits
    assert ab("mid_fwd") == ab("mid_inv") == 2 * pairs * slot
    assert ab("prep") == nkeys * 8
    assert ab("unknown") == 0


def test_workload_is_the_dv_qkd_set():
    assert bench.subconfigs() == [(1_000_000, 100_000), (1_000_000, 250_000), (1_000_000, 500_000),
                                  (1 << 20, 104_857), (1 << 20, 262_144), (1 << 20, 524_288)]
    assert bench.NKEYS == 64


def test_long_block_pass_bytes_and_work():
    n, m, L = 1 << 27, 1 << 24, 9 << 24  # L = 150,994,944: a lone key in N = L/2 complex values
    W = 8 * (L // 2)                     # 603,979,776 bytes of work slot
    b = bench.long_block_pass_bytes(L, n, m)
    assert b["fwd_keys"] == W + n // 8 == 620_756_992      # key bits in, W out
    assert b["mid_fwd"] == b["mid_inv"] == 2 * W          # W in and out
    assert b["middle_conv"] == 5 * W == 3_019_898_880     # W in, three seed tables, W out
    assert b["inv_bits"] == W + m // 8 == 606_076_928      # W in, final key out
    assert 20 * L + (n + m) // 8 == 3_038_773_248          # the FP32 path's floor per block
    # NTT64: L = 2^28, one transform each way (N/2 log2 N products) plus the pointwise product
    work, unit = bench.long_block_work("ntt64", 1 << 28)
    assert unit == "modmul" and work == 2 * (1 << 27) * 28 + (1 << 28) == 29 << 28
    # FP64: half-length form, two complex transforms of N points (5 N log2 N flops each), 38 per bin
    work, unit = bench.long_block_work("fp64", L)
    N = L // 2
    assert unit == "flop" and abs(work - (10 * N * math.log2(N) + 38 * N)) < 1e-3 * work

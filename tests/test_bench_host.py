"""Host-side arithmetic of bench.py (no GPU): the per-launch algorithmic bytes behind the
roofline's `achieved` figure, written out by hand for the DV-QKD batch n = 2^20, m = 2^18
(L = 5 * 2^18, 32 key pairs, 64 keys, FP32 slots of 8 bytes per complex value)."""
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

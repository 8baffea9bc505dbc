"""Benchmark: PA input Mbit/s of the FFT Toeplitz hash on one GB300 (bit-exact path).

Workload (the DV-QKD block sizes): n in {1,000,000, 2^20} input bits x
compression m/n in {0.1, 0.25, 0.5}; for each of the six (n, m) pairs, a batch
of 64 independent keys that share one Toeplitz seed (its spectrum cached on the
device). One step hashes all six batches, FP32 transforms with the per-key
rounding guard (escalating to FP64 when the margin exceeds 0.25). Inputs are
i.i.d. Bernoulli(0.5) bits (SplitMix64, seed 0), already resident in HBM.

Reported beside the headline: the plain single-key FP64 form on the same
sizes, p50/p99 batch latency, the dominant kernel's roofline, an end-to-end
number through host buffers, and the CPU oracle on a bounded sample.

``--impl reference`` times the CPU oracle instead (the reference arm).
Under torchrun (N > 1) every rank hashes its own batches (replicas; the path
has no exchange step) and rank 0 prints the whole-job number.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "dv_qkd_64keys_shared_seed"
N_VALUES = (1_000_000, 1 << 20)
RATIOS = (0.1, 0.25, 0.5)
NKEYS = 64
METRIC = "PA input Mbit/s per GB300 (bit-exact), batched/FP32 vs plain FP64; p50/p99 block latency"


def subconfigs():
    return [(n, int(r * n)) for n in N_VALUES for r in RATIOS]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# The files that define the pass kernels, their launch shapes and the transform splits;
# an ncu summary's DRAM figures hold while these are unchanged.
KERNEL_SOURCES = ("fft_core.cuh", "pa_kernels.cuh", "bulk.cuh", "zp.cuh", "pa_launch.h", "pa_launch.cuh",
                  "pa_geometry.cu", "pa_f32.cu", "pa_f32_r3.cu", "pa_f32_r5.cu", "pa_f32_r9.cu")


def source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1809_07592_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if its source hash is current."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{WORKLOAD}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if ":" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(kind: str, n: int, m: int, L: int, pairs: int, nkeys: int, elem: int) -> float:
    """Compulsory bytes one launch of a kernel family moves (complex work slot = L * elem bytes per pair)."""
    slot = L * elem
    kw, ow = (n + 63) // 64 * 8, (m + 63) // 64 * 8
    if kind == "fwd_keys":
        return pairs * slot + nkeys * kw
    if kind == "middle_conv":
        return 2 * pairs * slot + slot  # W in, W out, seed spectrum once
    if kind == "inv_bits":
        return pairs * slot + nkeys * ow
    if kind in ("mid_fwd", "mid_inv"):
        return 2 * pairs * slot
    if kind == "prep":
        return nkeys * 8  # popcount and margin words reset
    return 0.0


def workload_config(world: int) -> dict:
    """The workload both arms report (the reference arm runs a bounded sample of it)."""
    return {"workload": WORKLOAD, "n": list(N_VALUES), "m_over_n": list(RATIOS), "keys_per_batch": NKEYS,
            "batches_per_step": len(subconfigs()), "mode": "FP32_GUARD",
            "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas{world}"}


def _oracle_key(oracle, inputs, threads, batch, key_index):
    """The oracle on the whole of key `key_index` of batch `batch` of the workload (the same seed and
    key as the GPU step), every row. Returns (key bits, seconds)."""
    n, m = subconfigs()[batch]
    seed = inputs.bernoulli_bits(0, inputs.STREAM_SEED, n + m - 1)
    key = inputs.batch_keys(n, 1, base_seed=0, first_stream=2 + key_index)[0]  # key key_index of the batch
    t0 = time.perf_counter()
    oracle.toeplitz_hash(n, m, seed, key, threads)
    return n, time.perf_counter() - t0


def _oracle_keys(oracle, inputs, threads, key_index):
    """Whole key `key_index` of each of the six (n, m) batches. Returns (key bits, seconds)."""
    bits, secs = 0, 0.0
    for b in range(len(subconfigs())):
        nb, sb = _oracle_key(oracle, inputs, threads, b, key_index)
        bits += nb
        secs += sb
    return bits, secs


def cpu_baseline(budget_s: float = 12.0):
    """The oracle, as it stands, on a bounded sample of the workload: whole keys of the six (n, m)
    batches (key 0 of each, then key 1, ...) until about budget_s seconds of CPU work."""
    from oracle import oracle
    from paper_1809_07592_gb300 import inputs
    threads = os.cpu_count() or 1
    bits, secs, k = 0, 0.0, 0
    while secs < budget_s and k < NKEYS:
        b, t = _oracle_keys(oracle, inputs, threads, k)
        bits += b
        secs += t
        k += 1
    return {"value": bits / secs / 1e6, "unit": "Mbit/s", "cores": threads, "kind": "oracle",
            "sample": f"keys 0..{k - 1} of each of the six (n, m) batches, every row, in {secs:.2f} s",
            "seconds": round(secs, 3)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle
    from paper_1809_07592_gb300 import inputs
    threads = os.cpu_count() or 1
    nb = len(subconfigs())
    # every step hashes one whole key, every row, with the oracle: step s takes key s // 6 of
    # batch s % 6, so consecutive steps walk through the six (n, m) batches; the warm-up steps
    # (which also build the oracle) take keys from the other end of each batch
    for w in range(args.warmup):
        _oracle_key(oracle, inputs, threads, w % nb, NKEYS - 1 - (w // nb) % NKEYS)
    times, bits = [], 0
    for s in range(args.steps):
        b, t = _oracle_key(oracle, inputs, threads, s % nb, (s // nb) % NKEYS)
        bits += b
        times.append(t)
    total = sum(times)
    value = bits / total / 1e6
    line = {"metric": METRIC, "value": value, "unit": "Mbit/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(world), "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": threads, "value": value, "unit": "Mbit/s",
                             "sample": "one whole key (every row) per step: step s hashes key s // 6 of the "
                                       "(n, m) batch s % 6", "seconds": round(total, 3)},
            "e2e": {"value": value, "unit": "Mbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _dev_words(torch, words, device):
    w = np.zeros(words.size + (words.size & 1), dtype=np.uint64)
    w[: words.size] = words
    return torch.from_numpy(w.view(np.int64)).to(device)


def measure_uneven(pa, inputs, torch, dev, reps=5):
    """256 blocks, n log-uniform in [2^16, 2^24], m/n in [0.05, 0.6], per-block seeds, graph replay."""
    sizes = inputs.uneven_sizes(256, base_seed=0)
    blocks = []
    for b, (n, m) in enumerate(sizes):
        k = _dev_words(torch, inputs.bernoulli_bits(0, 2 * b + 2, n), dev)
        sd = _dev_words(torch, inputs.bernoulli_bits(0, 2 * b + 3, n + m - 1), dev)
        ow = (m + 63) // 64
        blocks.append((n, m, k, sd, torch.empty(ow + (ow & 1), dtype=torch.int64, device=dev)))
    h = pa.pa_uneven_create(blocks, pa.PA_FP32_GUARD, use_graph=True)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        pa.pa_uneven_run(h, len(blocks), stream)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pa.pa_uneven_run(h, len(blocks), stream)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    classes = pa.pa_uneven_classes(h)
    pa.pa_uneven_destroy(h)
    bits = sum(n for n, _ in sizes)
    return {"value": bits / (ms * 1e-3) / 1e6, "unit": "Mbit/s", "ms_per_batch": ms, "blocks": len(sizes),
            "mode": "FP32_GUARD", "graph": True,
            "classes": [{"L": c[0], "split": [c[1], c[2], c[3]], "blocks": c[4]} for c in classes]}


def measure_serving(pa, inputs, torch, dev, rate=5000.0, seconds=1.0):
    """Poisson arrivals, n from {2^18, 1e6, 2^22, 2^24} w.p. {0.4, 0.3, 0.2, 0.1}, m/n in [0.1, 0.5], 40 GB cap."""
    pool = {}
    for n in inputs.SERVE_N_CHOICES:
        pool[n] = []
        for j in range(8):
            k = _dev_words(torch, inputs.bernoulli_bits(9, 2 * j + 2, n), dev)
            sd = _dev_words(torch, inputs.bernoulli_bits(9, 2 * j + 3, n + n // 2), dev)
            pool[n].append((k, sd, torch.empty((n // 2 + 63) // 64 + 2, dtype=torch.int64, device=dev)))
    srv = pa.pa_server_create(hbm_cap_bytes=40 * 10**9, dtype=pa.PA_FP32_GUARD)
    warm = [pa.pa_submit(srv, n, n // 4, *pool[n][0]) for n in inputs.SERVE_N_CHOICES]
    for t in warm:
        pa.pa_wait(srv, t, 60000)
    count = int(rate * seconds)
    times, sizes = inputs.serving_requests(count, rate, base_seed=1)
    t0 = time.perf_counter()
    tickets = []
    for i, (t, (n, m)) in enumerate(zip(times, sizes)):
        while time.perf_counter() - t0 < t:
            pass
        tickets.append(pa.pa_submit(srv, n, m, *pool[n][i % 8]))
    submit_s = time.perf_counter() - t0
    res = [pa.pa_wait(srv, t, 120000) for t in tickets]
    st = pa.pa_server_stats(srv)
    pa.pa_server_destroy(srv)
    lat = np.array([(r.t_done_ns - r.t_submit_ns) / 1e6 for r in res])
    queue = np.array([(r.t_admit_ns - r.t_submit_ns) / 1e6 for r in res])  # waiting for admission
    run = np.array([(r.t_done_ns - r.t_admit_ns) / 1e6 for r in res])      # admitted until done
    span = (max(r.t_done_ns for r in res) - min(r.t_submit_ns for r in res)) / 1e9
    bits = sum(n for n, _ in sizes)
    pct = lambda a: {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "max": float(a.max())}
    return {"value": bits / span / 1e6, "unit": "Mbit/s", "offered_mbit_s": bits / times[-1] / 1e6,
            "arrival_rate_per_s": rate, "requests": count, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "queue_ms": pct(queue), "admitted_to_done_ms": pct(run),
            "submit_loop_s": submit_s, "arrival_span_s": float(times[-1]),
            "hbm_cap_bytes": 40 * 10**9,
            "peak_inflight_bytes": st["peak_inflight_bytes"], "micro_batches": st["batches"],
            "escalated": st["escalated"], "mode": "FP32_GUARD"}


def measure_cufft_comparison(pa, inputs, torch, dev, reps=10):
    """Comparison point only (not the product): the same DV-QKD step written with torch.fft (cuFFT)
    and torch elementwise ops -- bit unpack, real FFT of the 64 keys, product with the cached seed
    spectrum, inverse real FFT, rounding, parity, bit pack -- at the library's transform lengths, with
    the same +-1 seed encoding. Output bits of key 0 of every batch are checked against the library."""
    stream = torch.cuda.current_stream()
    shifts = torch.arange(64, device=dev, dtype=torch.int64)
    weights = (2 ** torch.arange(8, device=dev, dtype=torch.int32)).to(torch.uint8)
    cases = []
    for n, m in subconfigs():
        seed = inputs.bernoulli_bits(0, inputs.STREAM_SEED, n + m - 1)
        keys = inputs.batch_keys(n, NKEYS, base_seed=0)
        plan = pa.Plan(n, m, pa.PA_FP32_GUARD)
        L = plan.shape()[0]
        sd = _dev_words(torch, seed, dev)
        plan.set_seed(sd)
        kw = keys.shape[1] + (keys.shape[1] & 1)
        kb = np.zeros((NKEYS, kw), np.uint64)
        kb[:, : keys.shape[1]] = keys
        dk = torch.from_numpy(kb.view(np.int64)).to(dev)
        ow = (m + 63) // 64
        ref = plan.hash(dk)[:1, :ow].clone()
        plan.close()
        sbits = ((torch.from_numpy(seed.view(np.int64)).to(dev).unsqueeze(-1) >> shifts) & 1).flatten()[: n + m - 1]
        sigma = torch.zeros(L, device=dev, dtype=torch.float32)
        sigma[: n + m - 1] = 1.0 - 2.0 * sbits.to(torch.float32)
        S = torch.fft.rfft(sigma)
        cases.append(dict(n=n, m=m, L=L, dk=dk, S=S, ref=ref, ow=ow))

    def one(c):
        n, m, L = c["n"], c["m"], c["L"]
        x = ((c["dk"].unsqueeze(-1) >> shifts) & 1).flatten(1)[:, :n].to(torch.float32)  # 0/1 key bits
        r = torch.fft.irfft(torch.fft.rfft(x, n=L) * c["S"], n=L)[:, n - 1: n - 1 + m]  # r = P - 2c
        P = x.sum(dim=1, keepdim=True)
        y = torch.remainder(torch.round((P - r) * 0.5), 2.0).to(torch.uint8)
        pad = torch.zeros((NKEYS, c["ow"] * 64), device=dev, dtype=torch.uint8)
        pad[:, :m] = y
        packed = (pad.view(NKEYS, -1, 8) * weights).sum(dim=-1, dtype=torch.uint8)
        return packed.view(torch.int64)

    ok = all(torch.equal(one(c)[:1], c["ref"]) for c in cases)
    for _ in range(3):
        for c in cases:
            one(c)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for c in cases:
            one(c)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    # the transforms alone (keys already unpacked to floats): rfft, product, irfft
    xs = [((c["dk"].unsqueeze(-1) >> shifts) & 1).flatten(1)[:, : c["n"]].to(torch.float32) for c in cases]
    tf = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for c, x in zip(cases, xs):
            torch.fft.irfft(torch.fft.rfft(x, n=c["L"]) * c["S"], n=c["L"])
        b.record(stream)
        torch.cuda.synchronize()
        tf.append(a.elapsed_time(b))
    bits = sum(c["n"] for c in cases) * NKEYS
    return {"value": bits / (ms * 1e-3) / 1e6, "unit": "Mbit/s", "ms_per_step": ms, "bits_match_library": ok,
            "transforms_only_ms_per_step": statistics.median(tf),
            "form": "torch.fft (cuFFT) real transforms + torch elementwise ops, comparison point only"}


def measure_single_block(pa, inputs, torch, dev, reps=20):
    """The plain single block: n = 131072, m = 32768, one key, seed spectrum resident, FP64 and FP32_GUARD."""
    n, m = 131072, 32768
    key, seed = inputs.block_inputs(n, m, base_seed=0)
    kd, sd = _dev_words(torch, key, dev), _dev_words(torch, seed, dev)
    ow = (m + 63) // 64
    out = torch.empty((1, ow + (ow & 1)), dtype=torch.int64, device=dev)
    res = {}
    stream = torch.cuda.current_stream()
    for name, dt in (("fp64", pa.PA_FP64), ("fp32_guard", pa.PA_FP32_GUARD)):
        plan = pa.Plan(n, m, dt)
        plan.set_seed(sd)
        for _ in range(3):
            pa.pa_hash_batch(plan.handle, kd.view(1, -1), 1, kd.numel(), out, out.shape[1], stream)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pa.pa_hash_batch(plan.handle, kd.view(1, -1), 1, kd.numel(), out, out.shape[1], stream)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        res[name] = {"value": n / (ms * 1e-3) / 1e6, "unit": "Mbit/s", "ms": ms}
        plan.close()
    return res


def long_block_work(mode: str, L: int) -> tuple:
    """Algorithmic arithmetic of one long-block hash (one key) by the textbook counts: a
    complex FFT of N points costs 5 N log2 N flops, an exact NTT of N points N/2 log2 N
    modular products (radix-2 butterflies). FP64: a lone key runs in the half-length form,
    N = L/2: forward and inverse transforms plus the per-bin split and product with the
    three seed tables (38 flops per bin). NTT64: one transform of N = L points each way
    plus the pointwise product. Returns (amount, unit)."""
    import math
    if mode == "fp64":
        N = L // 2
        return 2 * 5 * N * math.log2(N) + 38 * N, "flop"
    N = L
    return 2 * (N / 2) * math.log2(N) + N, "modmul"


def long_block_pass_bytes(L: int, n: int, m: int) -> dict:
    """Bytes each pass of a single-key (half-length, N = L/2, W = 8 N bytes) FP32 block must move."""
    W = 8 * (L // 2)
    return {"fwd_keys": W + n / 8, "mid_fwd": 2 * W, "middle_conv": 5 * W, "mid_inv": 2 * W, "inv_bits": W + m / 8}


def long_block_passes(pa, plan, kd, out, stream, torch, n, m, block_ms, reps=5):
    """Per-pass roofline of the FP32 long block (one key, half-length form, N = L/2 complex values,
    W = 8 N bytes): each pass's live CUDA-event time (the library's per-launch events, in runs kept
    apart from the timed ones) against the bytes that pass must move -- first pass W + n/8, each
    middle strided pass 2 W, the fused innermost pass W in, the three seed tables (3 W) and W out,
    the last pass W + m/8 -- and the block against the FP32 path's floor of 20 L + (n+m)/8 bytes."""
    L = plan.shape()[0]
    need = long_block_pass_bytes(L, n, m)
    peak, kind = measured_peaks()
    pa.pa_profile_enable(plan.handle, True)
    pa.pa_profile_read(plan.handle, reset=True)
    for _ in range(reps):
        pa.pa_hash_batch(plan.handle, kd.view(1, -1), 1, kd.numel(), out, out.shape[1], stream)
    torch.cuda.synchronize()
    stats = pa.pa_profile_read(plan.handle, reset=True)
    pa.pa_profile_enable(plan.handle, False)
    passes = {}
    for k, b in need.items():
        cnt, tot = stats.get(k, (0, 0.0))
        if cnt:
            ms = tot / cnt
            gbs = b / (ms * 1e-3) / 1e9
            passes[k] = {"ms": ms, "bytes": b, "gbs": gbs, "frac": gbs / peak}
    floor = 20 * L + (n + m) / 8
    return {"per_pass": passes, "peak_gbs": peak, "peak_source": kind,
            "block_floor_bytes": floor, "block_floor_frac": floor / (block_ms * 1e-3) / 1e9 / peak,
            "block_design_bytes": sum(need.values()),
            "block_design_frac": sum(need.values()) / (block_ms * 1e-3) / 1e9 / peak}


def measure_long_block(pa, inputs, torch, dev, reps=3):
    """n = 2^27, m = 2^24 (transform length up to 2^28), one block, seed spectrum resident, per mode;
    the FP64 and NTT64 modes also against the measured FP64 FMA and modular-product peaks."""
    n, m = 1 << 27, 1 << 24
    key, seed = inputs.block_inputs(n, m, base_seed=0)
    kd, sd = _dev_words(torch, key, dev), _dev_words(torch, seed, dev)
    ow = (m + 63) // 64
    out = torch.empty((1, ow + (ow & 1)), dtype=torch.int64, device=dev)
    res = {}
    stream = torch.cuda.current_stream()
    for name, dt in (("fp32_guard", pa.PA_FP32_GUARD), ("fp64", pa.PA_FP64), ("ntt64", pa.PA_NTT64)):
        plan = pa.Plan(n, m, dt)
        plan.set_seed(sd)
        pa.pa_hash_batch(plan.handle, kd.view(1, -1), 1, kd.numel(), out, out.shape[1], stream)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pa.pa_hash_batch(plan.handle, kd.view(1, -1), 1, kd.numel(), out, out.shape[1], stream)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        res[name] = {"value": n / (ms * 1e-3) / 1e6, "unit": "Mbit/s", "ms": ms, "L": plan.shape()[0]}
        if name == "fp32_guard":
            res[name]["passes"] = long_block_passes(pa, plan, kd, out, stream, torch, n, m, ms)
        plan.close()
    fp64_gflops, zp_gmul = pa.pa_alu_peaks()
    for name, peak, unit in (("fp64", fp64_gflops * 1e9, "flop"), ("ntt64", zp_gmul * 1e9, "modmul")):
        work, u = long_block_work(name, res[name]["L"])
        rate = work / (res[name]["ms"] * 1e-3)
        res[name]["roofline"] = {"bound": "alu", "work": work, "work_unit": u, "achieved_per_s": rate,
                                 "peak_per_s": peak, "frac": rate / peak,
                                 "peak_source": "pa_alu_peaks (measured on this GPU in this run)"}
    return res


def measure_storage_precision(pa, inputs, torch, dev, bits_list=(23, 16, 13, 10, 7), lgs=range(16, 21), nkeys=8):
    """The paper's Section 5 precision question, measured: the FP32 path with every value stored
    between passes rounded to a narrower significand (pa_plan_set_storage_bits; 10 bits as in
    FP16, 7 as in BF16), guard off, n = 2^16 .. 2^20, m = n/4, 8 keys: the largest rounding margin
    max|w - rint(w)| over the keys. Above 0.25 the guard would send a key to FP64; near 0.5 the
    rounding error has reached a whole unit and the parity is noise."""
    table = {}
    for lg in lgs:
        n = 1 << lg
        m = n // 4
        seed = inputs.bernoulli_bits(lg, inputs.STREAM_SEED, n + m - 1)
        keys = inputs.batch_keys(n, nkeys, base_seed=lg)
        kw = keys.shape[1] + (keys.shape[1] & 1)
        kb = np.zeros((nkeys, kw), np.uint64)
        kb[:, : keys.shape[1]] = keys
        dk = torch.from_numpy(kb.view(np.int64)).to(dev)
        row = {}
        for bits in bits_list:
            plan = pa.Plan(n, m, pa.PA_FP32_GUARD)
            pa.pa_plan_set_storage_bits(plan.handle, bits)
            pa.pa_plan_set_guard(plan.handle, 1e9)
            plan.set_seed(_dev_words(torch, seed, dev))
            _, (marg, _mode, _esc) = plan.hash(dk, info=True)
            torch.cuda.synchronize()
            plan.close()
            row[str(bits)] = max(marg)
        table[str(n)] = row
    return {"margin_max_by_n_and_significand_bits": table, "m_over_n": 0.25, "keys": nkeys,
            "note": "guard off; 23 = FP32 storage as the product runs it"}


def measure_modified(pa, inputs, torch, dev, steps=20):
    """The modified Toeplitz hash [I_m, T'] (Eq. 2-3) on the same DV-QKD batches (64 keys per (n, m),
    one seed of n-1 bits each): one step issues the six batches, then runs their guard steps."""
    stream = torch.cuda.current_stream()
    cases = []
    for n, m in subconfigs():
        seed = inputs.bernoulli_bits(0, inputs.STREAM_SEED, n - 1)
        keys = inputs.batch_keys(n, NKEYS, base_seed=0)
        kw = keys.shape[1] + (keys.shape[1] & 1)
        kb = np.zeros((NKEYS, kw), np.uint64)
        kb[:, : keys.shape[1]] = keys
        ow = (m + 63) // 64
        ow += ow & 1
        plan = pa.Plan(n, m, pa.PA_FP32_GUARD, modified=True)
        plan.set_seed(_dev_words(torch, seed, dev))
        cases.append(dict(n=n, plan=plan, kw=kw, ow=ow, dk=torch.from_numpy(kb.view(np.int64)).to(dev),
                          out=torch.empty((NKEYS, ow), dtype=torch.int64, device=dev)))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step():
        for c in cases:
            pa.pa_hash_batch_async(c["plan"].handle, c["dk"], NKEYS, c["kw"], c["out"], c["ow"], stream)
        for c in cases:
            pa.pa_batch_finish(c["plan"].handle)

    for _ in range(3):
        step()
    ts = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.mean(ts)
    bits = sum(c["n"] for c in cases) * NKEYS
    res = {"value": bits / (ms * 1e-3) / 1e6, "unit": "Mbit/s", "ms_per_step": ms, "mode": "FP32_GUARD",
           "transform_lengths": [c["plan"].shape()[0] for c in cases]}
    for c in cases:
        c["plan"].close()
    return res


def run_ours(args):
    import torch
    import paper_1809_07592_gb300 as pa
    from paper_1809_07592_gb300 import inputs, replicas

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    pa.lib()

    # --- inputs resident in HBM; one plan + seed per (n, m) -------------------------------------------
    cases = []
    base = replicas.rank_base_seed(rank)  # each replica draws its own keys
    for n, m in subconfigs():
        seed = inputs.bernoulli_bits(base, inputs.STREAM_SEED, n + m - 1)
        keys = inputs.batch_keys(n, NKEYS, base_seed=base)
        kw = keys.shape[1] + (keys.shape[1] & 1)
        kb = np.zeros((NKEYS, kw), np.uint64)
        kb[:, : keys.shape[1]] = keys
        sw = np.zeros(seed.size + (seed.size & 1), np.uint64)
        sw[: seed.size] = seed
        ow = (m + 63) // 64
        ow += ow & 1
        plan = pa.Plan(n, m, pa.PA_FP32_GUARD)
        plan.set_seed(torch.from_numpy(sw.view(np.int64)).to(dev))
        dk = torch.from_numpy(kb.view(np.int64)).to(dev)
        out = torch.empty((NKEYS, ow), dtype=torch.int64, device=dev)
        hk = torch.from_numpy(kb.view(np.int64)).pin_memory()
        ho = torch.empty((NKEYS, ow), dtype=torch.int64).pin_memory()
        cases.append(dict(n=n, m=m, plan=plan, dk=dk, out=out, hk=hk, ho=ho, kw=kw, ow=ow, seed_dev=sw))
    # issue order within a step: outputs largest first, so the batch whose final keys are copied
    # back last has the fewest of them
    issue = sorted(cases, key=lambda c: -c["m"])
    lengths = [c["plan"].shape()[0] for c in cases]
    splits = [list(c["plan"].shape()[1:]) for c in cases]  # chosen by the plan's split autotuner
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    # The batches of a step alternate between two streams: while one batch's short tail
    # launches drain, the next batch's first pass already fills the SMs.
    sides = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]

    def join_sides():
        for sd in sides:
            stream.wait_stream(sd)

    def step(end_event=None, overlap=True):
        # Every batch is issued before the first guard step runs, so the GPU sees the six
        # batches back to back (batch i on side stream i % 2, both after the main stream's
        # work so far). end_event is recorded on the main stream behind every batch (its kernels
        # and margin read-back); the guard steps then run on the host. If a guard recomputes
        # any key, that work is issued after end_event, so the step then ends at an event
        # recorded behind it (returned as the second value). overlap=False keeps every batch on
        # one stream, so that per-launch events time each kernel alone.
        for sd in sides:
            sd.wait_stream(stream)
        lat = []
        for i, c in enumerate(issue):
            sd = sides[i % 2] if overlap else sides[0]
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(sd)
            pa.pa_hash_batch_async(c["plan"].handle, c["dk"], NKEYS, c["kw"], c["out"], c["ow"], sd)
            b.record(sd)
            lat.append((a, b))
        join_sides()
        if end_event is not None:
            end_event.record(stream)
        escalated = 0
        for c in cases:
            escalated += pa.pa_batch_finish(c["plan"].handle, NKEYS, info=True)[2]
        join_sides()
        late_end = None
        if escalated and end_event is not None:
            late_end = torch.cuda.Event(enable_timing=True)
            late_end.record(stream)
        return lat, late_end

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()

    step_ms, lat_ms = [], []
    torch.cuda.profiler.start()  # a profiler run with --profile-from-start off sees the timed steps only
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            lat, late_end = step(s1)
            torch.cuda.synchronize()
            step_ms.append(s0.elapsed_time(late_end if late_end is not None else s1))
            lat_ms += [a.elapsed_time(b) for a, b in lat]
    torch.cuda.profiler.stop()
    barrier()

    # per-kernel timings: the same steps again with the library's per-launch CUDA events on
    # (kept out of the timed steps above, whose rate they would lower)
    for c in cases:
        pa.pa_profile_enable(c["plan"].handle, True)
        pa.pa_profile_read(c["plan"].handle, reset=True)
    prof_steps = max(3, min(args.steps, 50))
    for _ in range(prof_steps):
        flush.zero_()
        barrier()
        step(overlap=False)
    barrier()
    prof = {}
    for c in cases:
        for k, (cnt, ms) in pa.pa_profile_read(c["plan"].handle, reset=True).items():
            pc = prof.setdefault(k, [0, 0.0, 0.0])
            pc[0] += cnt
            pc[1] += ms
            if cnt:
                shape = c["plan"].shape()
                pc[2] += cnt * algorithmic_bytes(k, c["n"], c["m"], shape[0], NKEYS // 2, NKEYS, 8)
        pa.pa_profile_enable(c["plan"].handle, False)
    # library kernels per step (from the profiled steps) times the timed steps
    gpu_launches = int(round(sum(v[0] for v in prof.values()) / prof_steps * args.steps))
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_cnt, dom_ms, dom_bytes) = dom
    avg_ms = dom_ms / dom_cnt
    achieved = (dom_bytes / dom_cnt) / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = ncu_traffic(dom_name)

    bits_per_step = sum(c["n"] for c in cases) * NKEYS
    t_max = replicas.max_over_ranks(statistics.mean(step_ms), dev)
    value = replicas.whole_job_rate(bits_per_step, world, t_max * 1e-3) / 1e6

    # --- plain single-key FP64 form on the same sizes (the other side of the metric) ---------------
    fp64 = []
    for c in cases:
        p64 = pa.Plan(c["n"], c["m"], pa.PA_FP64)
        p64.set_seed(torch.from_numpy(c["seed_dev"].view(np.int64)).to(dev))
        o1 = torch.empty((1, c["ow"]), dtype=torch.int64, device=dev)
        pa.pa_hash_batch(p64.handle, c["dk"][0:1], 1, c["kw"], o1, c["ow"])
        torch.cuda.synchronize()
        ts = []
        for k in range(4):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pa.pa_hash_batch(p64.handle, c["dk"][k:k + 1], 1, c["kw"], o1, c["ow"])
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        fp64.append((c["n"], statistics.median(ts)))
        p64.close()
    fp64_value = sum(n for n, _ in fp64) / (sum(t for _, t in fp64) * 1e-3) / 1e6

    # --- end to end through host buffers: pa_hash_host_async copies each batch's keys in from pinned
    # host memory and its final keys back, on copy streams that overlap the other batches' compute;
    # pa_batch_finish runs the guard (the host rows are final after it) ---------------------------
    h2d = sum(NKEYS * ((c["n"] + 63) // 64) * 8 for c in cases)
    d2h = sum(NKEYS * ((c["m"] + 63) // 64) * 8 for c in cases)
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for sd in sides:
            sd.wait_stream(stream)
        for i, c in enumerate(issue):
            pa.pa_hash_host_async(c["plan"].handle, c["hk"], NKEYS, c["kw"], c["ho"], c["ow"], sides[i % 2])
        for c in cases:
            pa.pa_batch_finish(c["plan"].handle)
        join_sides()
        s1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_ms.append(s0.elapsed_time(s1))
    te = replicas.max_over_ranks(statistics.mean(e2e_ms), dev)
    e2e_value = replicas.whole_job_rate(bits_per_step, world, te * 1e-3) / 1e6

    extra = {}
    if rank == 0 and not args.headline_only:
        extra["uneven_256_blocks"] = measure_uneven(pa, inputs, torch, dev)
        extra["serving"] = measure_serving(pa, inputs, torch, dev)
        extra["serving_rates"] = {}
        # below, at and past saturation: served Mbit/s levels off at the loop's capacity while the
        # admission wait (queue_ms) grows
        for rate in (200.0, 1000.0, 2000.0, 10000.0, 20000.0, 50000.0):
            secs = 2.0 if rate < 1000 else 1.0 if rate <= 10000 else 0.5
            sv = measure_serving(pa, inputs, torch, dev, rate=rate, seconds=secs)
            extra["serving_rates"][str(int(rate))] = {k: sv[k] for k in (
                "value", "offered_mbit_s", "p50_ms", "p99_ms", "max_ms", "requests", "queue_ms",
                "admitted_to_done_ms", "submit_loop_s", "arrival_span_s", "micro_batches")}
        extra["single_block_131072"] = measure_single_block(pa, inputs, torch, dev)
        extra["cufft_comparison"] = measure_cufft_comparison(pa, inputs, torch, dev)
        extra["long_block_2p27"] = measure_long_block(pa, inputs, torch, dev)
        extra["modified_toeplitz"] = measure_modified(pa, inputs, torch, dev)
        extra["storage_precision"] = measure_storage_precision(pa, inputs, torch, dev)

    if rank == 0:
        lat_sorted = sorted(lat_ms)
        p50 = float(np.percentile(lat_sorted, 50))
        p99 = float(np.percentile(lat_sorted, 99))
        line = {
            "metric": METRIC, "value": value, "unit": "Mbit/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(world),
            "plans": {"transform_lengths": lengths, "pass_splits": splits, "streams": len(sides)},
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
            "batch_latency_ms": {"p50": p50, "p99": p99, "unit": "ms per 64-key batch, two batches in flight"},
            "fp64_plain": {"value": fp64_value, "unit": "Mbit/s",
                           "form": "single key per call, FP64 transforms, same (n, m) set"},
            "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                         "avg_launch_ms": avg_ms, "launches": dom_cnt},
            "kernels": {k: {"launches": v[0], "avg_ms": v[1] / v[0] if v[0] else None,
                            "achieved_gbs": (v[2] / v[0]) / (v[1] / v[0] * 1e-3) / 1e9 if v[0] else None}
                        for k, v in prof.items() if v[0]},
            "gpu_launches": gpu_launches,
            "e2e": {"value": e2e_value, "unit": "Mbit/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "step_ms": {"min": min(e2e_ms), "median": statistics.median(e2e_ms), "max": max(e2e_ms)}},
            "clocks": clocks.summary(),
        }
        if "serving" in extra:
            sv = extra["serving"]
            line["latency_ms"] = {"p50": sv["p50_ms"], "p99": sv["p99_ms"],
                                  "unit": "ms per block, serving loop at 5000 blocks/s"}
        line.update(extra)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    for c in cases:
        c["plan"].close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true", help="skip the uneven, serving and long-block legs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

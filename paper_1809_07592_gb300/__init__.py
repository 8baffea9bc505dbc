"""GB300 FFT Toeplitz-hash privacy amplification: Python binding of libpa.so.

Thin ctypes marshalling over the C ABI in ``include/pa.h``. Every step of the
hash (bit unpacking, the FFT passes, the product with the seed spectrum,
rounding, parity and packing) runs in libpa.so's CUDA kernels; PyTorch only
provides device memory and streams. There is no CPU fallback: if libpa.so is
not built, or no CUDA device is present, these calls raise.

Names follow the C ABI: ``pa_plan``, ``pa_set_seed``, ``pa_hash_batch``, ...
A key tensor holds packed bits (bit j in 64-bit word j // 64 at position
j % 64); tensors are int64 on the device and reinterpreted as uint64.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

PA_OK = 0
PA_EINVAL = -1
PA_ENOMEM = -2
PA_EAGAIN = -3
PA_EPENDING = -4
PA_ETIMEOUT = -5
PA_EPRECISION = -6
PA_ECUDA = -7
PA_ENOSEED = -8
PA_EUNSUPPORTED = -9

PA_FP64 = 0
PA_FP32_GUARD = 1
PA_NTT64 = 2
DTYPES = {"fp64": PA_FP64, "fp32_guard": PA_FP32_GUARD, "fp32": PA_FP32_GUARD, "ntt64": PA_NTT64}

_lib = None


class PAError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {pa_strerror(code)}"
        if code == PA_ECUDA:
            msg += f" ({lib().pa_last_cuda_error().decode()})"
        super().__init__(msg)


class BatchInfo(ctypes.Structure):
    _fields_ = [("margin", ctypes.POINTER(ctypes.c_float)), ("mode", ctypes.POINTER(ctypes.c_int32)),
                ("escalated", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class BlockDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("m", ctypes.c_uint64), ("key", ctypes.c_void_p), ("seed", ctypes.c_void_p),
                ("out", ctypes.c_void_p)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_cap_bytes", ctypes.c_uint64), ("dtype", ctypes.c_int), ("max_queue", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("streams", ctypes.c_uint32), ("guard", ctypes.c_float)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("mode", ctypes.c_int32), ("margin", ctypes.c_float),
                ("reserved", ctypes.c_uint32), ("t_submit_ns", ctypes.c_uint64), ("t_admit_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "admitted", "completed", "escalated", "rejected",
                                               "batches", "queued", "inflight_bytes", "peak_inflight_bytes")]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


PA_NUM_KERNEL_KINDS = 8


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libpa.so (built in-tree by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libpa.so is not built at {path}; run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    L.pa_plan.argtypes = [u64, u64, ctypes.c_int, ctypes.POINTER(vp)]
    L.pa_plan_destroy.argtypes = [vp]
    L.pa_set_seed.argtypes = [vp, vp, u64, vp]
    L.pa_hash_batch.argtypes = [vp, vp, u32, u64, vp, u64, vp, ctypes.POINTER(BatchInfo)]
    L.pa_plan_set_guard.argtypes = [vp, ctypes.c_float]
    L.pa_plan_expire_waits.argtypes = [vp, u32]
    L.pa_plan_set_staged.argtypes = [vp, ctypes.c_int]
    L.pa_plan_set_storage_bits.argtypes = [vp, u32]
    L.pa_alu_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    L.pa_hash_batch_async.argtypes = [vp, vp, u32, u64, vp, u64, vp]
    L.pa_batch_finish.argtypes = [vp, ctypes.POINTER(BatchInfo)]
    L.pa_hash_host_async.argtypes = [vp, vp, u32, u64, vp, u64, vp]
    L.pa_hash_host.argtypes = [vp, vp, u32, u64, vp, u64, vp, ctypes.POINTER(BatchInfo)]
    L.pa_plan_shape.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u32), ctypes.POINTER(u32),
                                ctypes.POINTER(u32)]
    L.pa_plan_splits.argtypes = [u64, u64, ctypes.c_int, ctypes.POINTER(u32), ctypes.POINTER(u32),
                                 ctypes.POINTER(u32), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.pa_plan_split.argtypes = [u64, u64, ctypes.c_int, u32, u32, u32, ctypes.POINTER(vp)]
    L.pa_plan_modified.argtypes = [u64, u64, ctypes.c_int, ctypes.POINTER(vp)]
    L.pa_final_key_length.argtypes = [u64, u64, u64, ctypes.POINTER(u64)]
    L.pa_final_key_length.restype = ctypes.c_int
    L.pa_leakage_bound.argtypes = [u64, u64, u64]
    L.pa_leakage_bound.restype = ctypes.c_double
    L.pa_profile_enable.argtypes = [vp, ctypes.c_int]
    L.pa_profile_read.argtypes = [vp, ctypes.POINTER(KernelStat), ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    bdp = ctypes.POINTER(BlockDesc)
    L.pa_uneven_create.argtypes = [bdp, u32, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
    L.pa_uneven_update.argtypes = [vp, bdp, u32, vp]
    L.pa_uneven_run.argtypes = [vp, vp, ctypes.POINTER(BatchInfo)]
    L.pa_uneven_set_guard.argtypes = [vp, ctypes.c_float]
    L.pa_uneven_destroy.argtypes = [vp]
    L.pa_uneven_class.argtypes = [vp, u32, ctypes.POINTER(u32), ctypes.POINTER(u64), ctypes.POINTER(u32),
                                  ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
    L.pa_hash_uneven.argtypes = [bdp, u32, ctypes.c_int, vp, ctypes.POINTER(BatchInfo)]
    L.pa_server_create.argtypes = [ctypes.POINTER(ServerCfg), ctypes.POINTER(vp)]
    L.pa_submit.argtypes = [vp, bdp, ctypes.POINTER(u64)]
    L.pa_poll.argtypes = [vp, u64, ctypes.POINTER(Result)]
    L.pa_wait.argtypes = [vp, u64, u32, ctypes.POINTER(Result)]
    L.pa_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.pa_server_destroy.argtypes = [vp]
    L.pa_strerror.argtypes = [ctypes.c_int]
    L.pa_strerror.restype = ctypes.c_char_p
    L.pa_last_cuda_error.argtypes = []
    L.pa_last_cuda_error.restype = ctypes.c_char_p
    for name in ("pa_plan", "pa_plan_destroy", "pa_set_seed", "pa_hash_batch", "pa_hash_batch_async",
                 "pa_batch_finish", "pa_hash_host_async", "pa_hash_host", "pa_plan_set_guard",
                 "pa_plan_shape", "pa_plan_splits", "pa_plan_split", "pa_plan_modified", "pa_profile_enable", "pa_profile_read", "pa_uneven_create", "pa_uneven_update",
                 "pa_uneven_run", "pa_uneven_set_guard", "pa_uneven_destroy", "pa_uneven_class", "pa_hash_uneven",
                 "pa_server_create", "pa_submit", "pa_poll", "pa_wait", "pa_server_stats", "pa_server_destroy"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, where: str) -> None:
    if rc != PA_OK:
        raise PAError(rc, where)


def pa_strerror(code: int) -> str:
    return lib().pa_strerror(code).decode()


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr()


def pa_plan(n: int, m: int, dtype=PA_FP32_GUARD) -> int:
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    h = ctypes.c_void_p()
    _check(lib().pa_plan(n, m, dtype, ctypes.byref(h)), "pa_plan")
    return h.value


def pa_plan_splits(n: int, m: int, dtype=PA_FP32_GUARD):
    """The pass splits (L1, L2, L3) a plan of (n, m, dtype) chooses among."""
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    cnt = ctypes.c_int()
    _check(lib().pa_plan_splits(n, m, dtype, None, None, None, 0, ctypes.byref(cnt)), "pa_plan_splits")
    k = cnt.value
    a, b, c = (ctypes.c_uint32 * max(k, 1))(), (ctypes.c_uint32 * max(k, 1))(), (ctypes.c_uint32 * max(k, 1))()
    _check(lib().pa_plan_splits(n, m, dtype, a, b, c, k, ctypes.byref(cnt)), "pa_plan_splits")
    return [(a[i], b[i], c[i]) for i in range(k)]


def pa_plan_split(n: int, m: int, dtype, split) -> int:
    """pa_plan with the pass split fixed to one of pa_plan_splits' entries."""
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    h = ctypes.c_void_p()
    _check(lib().pa_plan_split(n, m, dtype, split[0], split[1], split[2], ctypes.byref(h)), "pa_plan_split")
    return h.value


def pa_final_key_length(n: int, t: int, s: int) -> int:
    """Eq. 1: final key length r = n - t - s for Eve's information t and security coefficient s."""
    r = ctypes.c_uint64()
    _check(lib().pa_final_key_length(n, t, s, ctypes.byref(r)), "pa_final_key_length")
    return r.value


def pa_leakage_bound(n: int, t: int, r: int) -> float:
    """Eq. 1: upper bound 2^-(n-t-r)/ln 2 on Eve's information about the r-bit final key."""
    return lib().pa_leakage_bound(n, t, r)


def pa_plan_modified(n: int, m: int, dtype=PA_FP32_GUARD) -> int:
    """Plan for the modified Toeplitz hash [I_m, T'] (keys of n bits, seeds of n-1 bits)."""
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    h = ctypes.c_void_p()
    _check(lib().pa_plan_modified(n, m, dtype, ctypes.byref(h)), "pa_plan_modified")
    return h.value


def pa_plan_destroy(plan: int) -> None:
    _check(lib().pa_plan_destroy(plan), "pa_plan_destroy")


def pa_plan_set_guard(plan: int, threshold: float) -> None:
    _check(lib().pa_plan_set_guard(plan, threshold), "pa_plan_set_guard")


def pa_plan_set_staged(plan: int, on: bool = True) -> None:
    """Run the plan's last pass as the TMA-staged persistent kernel (FP32, first pass <= 256)."""
    _check(lib().pa_plan_set_staged(plan, int(bool(on))), "pa_plan_set_staged")


def pa_plan_set_storage_bits(plan: int, bits: int) -> None:
    """Storage-precision study: keep `bits` significand bits of every value stored between passes."""
    _check(lib().pa_plan_set_storage_bits(plan, bits), "pa_plan_set_storage_bits")


def pa_plan_expire_waits(plan: int, launches: int = 1) -> None:
    """Test hook: the next `launches` pipelined convolution launches let their bounded wait run out."""
    _check(lib().pa_plan_expire_waits(plan, launches), "pa_plan_expire_waits")


def pa_alu_peaks(stream=None):
    """(FP64 GFLOP/s, G modular products/s) measured on the current device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().pa_alu_peaks(ctypes.byref(a), ctypes.byref(b), _stream_handle(stream)), "pa_alu_peaks")
    return a.value, b.value


def pa_plan_shape(plan: int):
    L = ctypes.c_uint64()
    a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().pa_plan_shape(plan, ctypes.byref(L), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "pa_plan_shape")
    return L.value, a.value, b.value, c.value


def pa_set_seed(plan: int, seed, seed_bits: int, stream=None) -> None:
    _check(lib().pa_set_seed(plan, _ptr(seed), seed_bits, _stream_handle(stream)), "pa_set_seed")


def pa_hash_batch(plan: int, keys, nkeys: int, key_stride_words: int, out, out_stride_words: int, stream=None,
                  info: bool = False):
    """Returns None, or (margins list, modes list, escalated) when ``info`` is set."""
    if info:
        marg = (ctypes.c_float * nkeys)()
        mode = (ctypes.c_int32 * nkeys)()
        bi = BatchInfo(ctypes.cast(marg, ctypes.POINTER(ctypes.c_float)),
                       ctypes.cast(mode, ctypes.POINTER(ctypes.c_int32)), 0, 0)
        _check(lib().pa_hash_batch(plan, _ptr(keys), nkeys, key_stride_words, _ptr(out), out_stride_words,
                                   _stream_handle(stream), ctypes.byref(bi)), "pa_hash_batch")
        return list(marg), list(mode), bi.escalated
    _check(lib().pa_hash_batch(plan, _ptr(keys), nkeys, key_stride_words, _ptr(out), out_stride_words,
                               _stream_handle(stream), None), "pa_hash_batch")
    return None


def pa_hash_batch_async(plan: int, keys, nkeys: int, key_stride_words: int, out, out_stride_words: int,
                        stream=None) -> None:
    """Issue a batch (kernels + margin read-back) without waiting; finish it with pa_batch_finish."""
    _check(lib().pa_hash_batch_async(plan, _ptr(keys), nkeys, key_stride_words, _ptr(out), out_stride_words,
                                     _stream_handle(stream)), "pa_hash_batch_async")


def _host_ptr(t) -> int:
    if t.is_cuda:
        raise ValueError("expected a host (CPU) tensor")
    return t.data_ptr()


def pa_hash_host_async(plan: int, keys, nkeys: int, key_stride_words: int, out, out_stride_words: int,
                       stream=None) -> None:
    """Host keys in, host final keys out (pinned CPU tensors overlap); finish with pa_batch_finish."""
    _check(lib().pa_hash_host_async(plan, _host_ptr(keys), nkeys, key_stride_words, _host_ptr(out), out_stride_words,
                                    _stream_handle(stream)), "pa_hash_host_async")


def pa_hash_host(plan: int, keys, nkeys: int, key_stride_words: int, out, out_stride_words: int, stream=None,
                 info: bool = False):
    """pa_hash_host_async + pa_batch_finish; (margins, modes, escalated) when ``info`` is set."""
    pa_hash_host_async(plan, keys, nkeys, key_stride_words, out, out_stride_words, stream)
    return pa_batch_finish(plan, nkeys, info)


def pa_batch_finish(plan: int, nkeys: int = 0, info: bool = False):
    """Guard step of an issued batch; (margins, modes, escalated) when ``info`` is set (nkeys needed)."""
    if info:
        marg = (ctypes.c_float * nkeys)()
        mode = (ctypes.c_int32 * nkeys)()
        bi = BatchInfo(ctypes.cast(marg, ctypes.POINTER(ctypes.c_float)),
                       ctypes.cast(mode, ctypes.POINTER(ctypes.c_int32)), 0, 0)
        _check(lib().pa_batch_finish(plan, ctypes.byref(bi)), "pa_batch_finish")
        return list(marg), list(mode), bi.escalated
    _check(lib().pa_batch_finish(plan, None), "pa_batch_finish")
    return None


def pa_profile_enable(plan: int, enable: bool = True) -> None:
    _check(lib().pa_profile_enable(plan, 1 if enable else 0), "pa_profile_enable")


def pa_profile_read(plan: int, reset: bool = False) -> dict:
    """{kernel family: (launches, total_ms)} accumulated since the last reset."""
    arr = (KernelStat * PA_NUM_KERNEL_KINDS)()
    cnt = ctypes.c_int()
    _check(lib().pa_profile_read(plan, arr, ctypes.byref(cnt), 1 if reset else 0), "pa_profile_read")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(cnt.value)}


def _descs(blocks):
    """blocks: iterable of (n, m, key_tensor, seed_tensor, out_tensor) -> ctypes array of BlockDesc."""
    blocks = list(blocks)
    arr = (BlockDesc * len(blocks))()
    for i, (n, m, k, sd, o) in enumerate(blocks):
        arr[i] = BlockDesc(n, m, _ptr(k), _ptr(sd), _ptr(o))
    return arr, len(blocks)


def _info_struct(nblocks):
    marg = (ctypes.c_float * nblocks)()
    mode = (ctypes.c_int32 * nblocks)()
    bi = BatchInfo(ctypes.cast(marg, ctypes.POINTER(ctypes.c_float)), ctypes.cast(mode, ctypes.POINTER(ctypes.c_int32)),
                   0, 0)
    return bi, marg, mode


def pa_uneven_create(blocks, dtype=PA_FP32_GUARD, use_graph: bool = True) -> int:
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    arr, nb = _descs(blocks)
    h = ctypes.c_void_p()
    _check(lib().pa_uneven_create(arr, nb, dtype, 1 if use_graph else 0, ctypes.byref(h)), "pa_uneven_create")
    return h.value


def pa_uneven_update(batch: int, blocks, stream=None) -> None:
    arr, nb = _descs(blocks)
    _check(lib().pa_uneven_update(batch, arr, nb, _stream_handle(stream)), "pa_uneven_update")


def pa_uneven_run(batch: int, nblocks: int, stream=None, info: bool = False):
    if info:
        bi, marg, mode = _info_struct(nblocks)
        _check(lib().pa_uneven_run(batch, _stream_handle(stream), ctypes.byref(bi)), "pa_uneven_run")
        return list(marg), list(mode), bi.escalated
    _check(lib().pa_uneven_run(batch, _stream_handle(stream), None), "pa_uneven_run")
    return None


def pa_uneven_set_guard(batch: int, threshold: float) -> None:
    _check(lib().pa_uneven_set_guard(batch, threshold), "pa_uneven_set_guard")


def pa_uneven_destroy(batch: int) -> None:
    _check(lib().pa_uneven_destroy(batch), "pa_uneven_destroy")


def pa_uneven_classes(batch: int):
    """[(L, L1, L2, L3, nblocks)] for every length class of the batch."""
    nc = ctypes.c_uint32()
    _check(lib().pa_uneven_class(batch, 0xFFFFFFFF, ctypes.byref(nc), None, None, None, None, None), "pa_uneven_class")
    out = []
    for c in range(nc.value):
        L = ctypes.c_uint64()
        a, b, d, nb = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().pa_uneven_class(batch, c, None, ctypes.byref(L), ctypes.byref(a), ctypes.byref(b), ctypes.byref(d),
                                     ctypes.byref(nb)), "pa_uneven_class")
        out.append((L.value, a.value, b.value, d.value, nb.value))
    return out


def pa_hash_uneven(blocks, dtype=PA_FP32_GUARD, stream=None, info: bool = False):
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    arr, nb = _descs(blocks)
    if info:
        bi, marg, mode = _info_struct(nb)
        _check(lib().pa_hash_uneven(arr, nb, dtype, _stream_handle(stream), ctypes.byref(bi)), "pa_hash_uneven")
        return list(marg), list(mode), bi.escalated
    _check(lib().pa_hash_uneven(arr, nb, dtype, _stream_handle(stream), None), "pa_hash_uneven")
    return None


def pa_server_create(hbm_cap_bytes: int = 0, dtype=PA_FP32_GUARD, max_queue: int = 0, max_batch: int = 0,
                     streams: int = 0, guard: float = 0.25) -> int:
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    cfg = ServerCfg(hbm_cap_bytes, dtype, max_queue, max_batch, streams, guard)
    h = ctypes.c_void_p()
    _check(lib().pa_server_create(ctypes.byref(cfg), ctypes.byref(h)), "pa_server_create")
    return h.value


def pa_submit(server: int, n: int, m: int, key, seed, out) -> int:
    """Queue one block; returns its ticket. Raises PAError (code PA_EAGAIN when the queue is full)."""
    d = BlockDesc(n, m, _ptr(key), _ptr(seed), _ptr(out))
    t = ctypes.c_uint64()
    _check(lib().pa_submit(server, ctypes.byref(d), ctypes.byref(t)), "pa_submit")
    return t.value


def pa_poll(server: int, ticket: int):
    """Result struct when done, None while pending."""
    r = Result()
    rc = lib().pa_poll(server, ticket, ctypes.byref(r))
    if rc == PA_EPENDING:
        return None
    _check(rc, "pa_poll")
    return r


def pa_wait(server: int, ticket: int, timeout_ms: int):
    r = Result()
    _check(lib().pa_wait(server, ticket, timeout_ms, ctypes.byref(r)), "pa_wait")
    return r


def pa_server_stats(server: int) -> dict:
    st = ServerStats()
    _check(lib().pa_server_stats(server, ctypes.byref(st)), "pa_server_stats")
    return {f: getattr(st, f) for f, _ in ServerStats._fields_}


def pa_server_destroy(server: int) -> None:
    _check(lib().pa_server_destroy(server), "pa_server_destroy")


class Plan:
    """Owns one pa_plan handle; a convenience wrapper over the functions above."""

    def __init__(self, n: int, m: int, dtype=PA_FP32_GUARD, split=None, modified: bool = False):
        self.n, self.m, self.modified = n, m, modified
        if modified:
            self.handle = pa_plan_modified(n, m, dtype)
        else:
            self.handle = pa_plan(n, m, dtype) if split is None else pa_plan_split(n, m, dtype, split)

    def seed_bits(self) -> int:
        return self.n - 1 if self.modified else self.n + self.m - 1

    def words_in(self) -> int:
        return (self.n + 63) // 64

    def words_out(self) -> int:
        return (self.m + 63) // 64

    def set_seed(self, seed, stream=None):
        pa_set_seed(self.handle, seed, self.seed_bits(), stream)

    def hash(self, keys, out=None, stream=None, info=False):
        """keys: (nkeys, stride) int64 CUDA tensor (stride even or nkeys == 1)."""
        import torch
        if keys.dim() == 1:
            keys = keys.view(1, -1)
        nkeys, kstride = keys.shape
        if out is None:
            ostride = self.words_out() + (self.words_out() & 1)
            out = torch.empty((nkeys, ostride), dtype=torch.int64, device=keys.device)
        r = pa_hash_batch(self.handle, keys, nkeys, kstride, out, out.shape[1], stream, info)
        return (out, r) if info else out

    def shape(self):
        return pa_plan_shape(self.handle)

    def close(self):
        if self.handle:
            pa_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pa_hash_static(n: int, m: int, dtype, seed, keys, nkeys: int, key_stride_words: int, out,
                   out_stride_words: int, stream=None) -> float:
    """Allocation-free hash of 1 or 2 keys (see pa_hash_static in pa.h); returns the rounding margin."""
    L = lib()
    if getattr(L.pa_hash_static, "_pa_typed", None) is None:
        u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        L.pa_hash_static.argtypes = [u64, u64, ctypes.c_int, vp, vp, u32, u64, vp, u64, vp,
                                     ctypes.POINTER(ctypes.c_float)]
        L.pa_hash_static.restype = ctypes.c_int
        L.pa_hash_static._pa_typed = True
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    marg = ctypes.c_float(0.0)
    _check(L.pa_hash_static(n, m, dtype, _ptr(seed), _ptr(keys), nkeys, key_stride_words, _ptr(out),
                            out_stride_words, _stream_handle(stream), ctypes.byref(marg)), "pa_hash_static")
    return marg.value

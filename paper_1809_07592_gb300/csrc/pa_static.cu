// pa_static.cu -- pa_hash_static: the hash of one or two keys without any
// device allocation.
//
// Some callers of this library cannot call cudaMalloc: a process whose device
// memory is entirely reserved by another framework's caching allocator, a
// real-time key-distillation loop that must not pay cudaMalloc's latency or
// the device-wide synchronisation of cudaFree, or an embedding that forbids
// dynamic allocation after start-up. pa_plan allocates its work buffers, so
// those callers use this entry point instead. All of its scratch -- the
// transform work slot, the seed spectrum, the twiddle tables and the per-key
// counters -- lives in one file-scope __device__ array of kScratchBytes bytes
// (65 MiB), which every GPU that loads the library holds until the process
// exits. Inputs and outputs stay caller-owned.
//
// The paper has no counterpart to this entry point; it is a deployment aid.
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>

#include <cuda.h>  // driver types of the context-id query (resolved at run time, no link to libcuda)

#include "pa.h"
#include "pa_launch.h"

using namespace pa;

namespace {

// Largest supported transform: complex length 2^21 (n + m - 1 <= 2^21, e.g. the
// n = 2^20, m <= n/2 blocks), two slots (work + spectrum) of FP64 complex values,
// plus twiddle tables and per-key counters.
constexpr int kMaxLgL = 21;
constexpr size_t kSlotBytes = ((size_t)1 << kMaxLgL) * 16;        // 32 MiB
constexpr size_t kScratchBytes = 2 * kSlotBytes + ((size_t)1 << 20);  // + 1 MiB tables and counters

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;

// Device address of g_scratch, per device, with the id of the context it belongs to.
// The address is valid only in that context: after cudaDeviceReset the module is
// loaded again into a new context (new id) and the address is looked up again.
struct ScratchAddr {
    unsigned char *ptr = nullptr;
    unsigned long long ctx = 0;
};
ScratchAddr g_scratch_addr[kMaxDevices];

// Unique id of the calling thread's current context (cuCtxGetCurrent + cuCtxGetId,
// resolved through the runtime's driver entry-point query); false if there is none.
bool current_context_id(unsigned long long *id) {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext c = nullptr;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_scratch on the current device: looked up (cudaGetSymbolAddress, with
// the device current) on the first call in a device's context, then taken from the cache.
int scratch_address(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PA_ECUDA;
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAddr &a = g_scratch_addr[dev];
    if (!have_id || !a.ptr || a.ctx != id) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return PA_ECUDA;
        a.ptr = static_cast<unsigned char *>(ptr);
        // the lookup made the device's primary context current if no context was
        unsigned long long now = 0;
        a.ctx = current_context_id(&now) ? now : 0;  // 0: no id, look up again next call
    }
    *out = a.ptr;
    return PA_OK;
}

// Guard threshold of pa_hash_static: 0.25, or the value of PA_STATIC_GUARD (a test sets
// it below every margin to drive the FP32 -> FP64 -> NTT64 recomputation).
float static_guard() {
    const char *s = std::getenv("PA_STATIC_GUARD");
    if (!s || !*s) return 0.25f;
    char *end = nullptr;
    const float v = std::strtof(s, &end);
    return (end && end != s) ? v : 0.25f;
}

// Twiddles of the complex transforms, exp(-2 pi i e / L) in double precision:
// the two-level table (hi, lo) and the stage table fine[j] = w_F^j, F = 2^lgF.
template <typename T>
__global__ void k_twiddles_complex(cx<T> *hi, cx<T> *lo, uint32_t B, uint32_t lgL, cx<T> *fine, uint32_t lgF) {
    const uint32_t nhi = 1u << (lgL - B), nlo = 1u << B, nf = 1u << lgF;
    const double inv = 1.0 / (double)(1ull << lgL);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nhi + nlo + nf; i += gridDim.x * blockDim.x) {
        double s, c;
        if (i < nhi + nlo) {
            const uint64_t e = i < nhi ? ((uint64_t)i << B) : (uint64_t)(i - nhi);
            sincospi(2.0 * (double)e * inv, &s, &c);
        } else {
            sincospi(2.0 * (double)(i - nhi - nlo) / (double)nf, &s, &c);
        }
        cx<T> w;
        w.x = (T)c;
        w.y = (T)-s;
        if (i < nhi) hi[i] = w; else if (i < nhi + nlo) lo[i - nhi] = w; else fine[i - nhi - nlo] = w;
    }
}

// w_L^e modulo p for the exact transform, by square-and-multiply from the root w;
// the stage table holds w_F^j = w_L^(j L/F).
__global__ void k_twiddles_zp(uint64_t *hi, uint64_t *lo, uint32_t B, uint32_t lgL, uint64_t w, uint64_t *fine,
                              uint32_t lgF) {
    const uint32_t nhi = 1u << (lgL - B), nlo = 1u << B, nf = 1u << lgF;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nhi + nlo + nf; i += gridDim.x * blockDim.x) {
        uint64_t e = i < nhi ? ((uint64_t)i << B)
                     : i < nhi + nlo ? (uint64_t)(i - nhi)
                                     : ((uint64_t)(i - nhi - nlo) << (lgL - lgF));
        uint64_t r = 1, b = w;
        while (e) {
            if (e & 1) r = zp_mul(r, b);
            b = zp_mul(b, b);
            e >>= 1;
        }
        if (i < nhi) hi[i] = r; else if (i < nhi + nlo) lo[i - nhi] = r; else fine[i - nhi - nlo] = r;
    }
}

uint64_t mulmod_host(uint64_t a, uint64_t b) {
    unsigned __int128 x = (unsigned __int128)a * b;
    return zp_reduce((uint64_t)(x >> 64), (uint64_t)x);
}
uint64_t powmod_host(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = mulmod_host(r, a);
        a = mulmod_host(a, a);
        e >>= 1;
    }
    return r;
}
// Root of order L whose L/32-th power is 2^6 (the in-register root), as in the plans.
uint64_t root_of_order(uint64_t L) {
    const uint64_t w = powmod_host(7, (kP - 1) / L);
    const uint64_t w32 = powmod_host(w, L / 32);
    for (uint64_t j = 1; j < 64; j += 2)
        if (powmod_host(w32, j) == 64ull) return powmod_host(w, j);
    return 0;
}

template <typename T> cx<T> scale_of(uint64_t L);
template <> cx<float> scale_of<float>(uint64_t L) { return make_float2((float)(1.0 / (double)L), 0.f); }
template <> cx<double> scale_of<double>(uint64_t L) { return make_double2(1.0 / (double)L, 0.0); }
template <> cx<Zp> scale_of<Zp>(uint64_t L) { return powmod_host(L, kP - 2); }
template <typename T> cx<T> unit();
template <> cx<float> unit<float>() { return make_float2(1.f, 0.f); }
template <> cx<double> unit<double>() { return make_double2(1.0, 0.0); }
template <> cx<Zp> unit<Zp>() { return 1ull; }

#define STATIC_CUDA(x)                               \
    do {                                             \
        if ((x) != cudaSuccess) return PA_ECUDA;     \
    } while (0)

// One complete hash of nkeys (1 or 2) keys, every buffer carved from g_scratch.
template <typename T>
int run_static(unsigned char *base, int lgL, uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *keys,
               uint32_t nkeys, uint64_t kstride, uint64_t *out, uint64_t ostride, cudaStream_t st) {
    const uint64_t L = 1ull << lgL;
    cx<T> *W = reinterpret_cast<cx<T> *>(base);
    cx<T> *spec = reinterpret_cast<cx<T> *>(base + kSlotBytes);
    unsigned char *tail = base + 2 * kSlotBytes;
    const uint32_t B = (uint32_t)(lgL + 1) / 2;
    cx<T> *hi = reinterpret_cast<cx<T> *>(tail);
    cx<T> *lo = hi + (1u << (lgL - B));
    int lg1 = lgL - 12;
    if (lg1 < kMinLgStrided) lg1 = kMinLgStrided;
    if (lg1 > kMaxLgStrided) lg1 = kMaxLgStrided;
    const int lg2 = lgL - lg1;  // <= 12 for lgL <= 21: always a two-level split
    const uint32_t lgF = (uint32_t)(lg1 > lg2 ? lg1 : lg2);  // stage table: lcm of the pass lengths
    cx<T> *fine = reinterpret_cast<cx<T> *>(tail + (64u << 10));  // after hi/lo (<= 48 KiB); <= 64 KiB
    uint32_t *popc = reinterpret_cast<uint32_t *>(tail + (512u << 10));
    uint32_t *marg = popc + 2;
    if constexpr (std::is_same<T, Zp>::value) {
        const uint64_t w = root_of_order(L);
        if (!w) return PA_EUNSUPPORTED;
        k_twiddles_zp<<<64, 256, 0, st>>>(reinterpret_cast<uint64_t *>(hi), reinterpret_cast<uint64_t *>(lo), B,
                                          (uint32_t)lgL, w, reinterpret_cast<uint64_t *>(fine), lgF);
    } else {
        k_twiddles_complex<T><<<64, 256, 0, st>>>(hi, lo, B, (uint32_t)lgL, fine, lgF);
    }
    STATIC_CUDA(cudaGetLastError());
    TwTab<T> tw;
    tw.hi = hi;
    tw.lo = lo;
    tw.B = B;
    tw.lgL = (uint32_t)lgL;
    tw.fine = fine;
    tw.F = 1u << lgF;
    STATIC_CUDA(launch_fwd_seed<T>(lg1, seed, n, m, W, L, tw, st));
    STATIC_CUDA(launch_middle<T>(1, lg2, 1, W, spec, L, 1, tw, scale_of<T>(L), st));
    STATIC_CUDA(launch_zero_keys(nkeys, popc, marg, st));  // the forward pass accumulates the popcounts
    STATIC_CUDA(launch_fwd_keys<T>(lg1, keys, nkeys, kstride, n, W, L, 1, tw, popc, st));
    STATIC_CUDA(launch_middle<T>(1, lg2, 0, W, spec, L, 1, tw, unit<T>(), st));
    STATIC_CUDA(launch_inv_bits<T>(lg1, W, L, m, nkeys, popc, marg, out, ostride, 1, tw, st));
    return PA_OK;
}

}  // namespace

extern "C" int pa_hash_static(uint64_t n, uint64_t m, pa_dtype_t dtype, const uint64_t *seed_dev,
                              const uint64_t *keys_dev, uint32_t nkeys, uint64_t key_stride_words,
                              uint64_t *out_dev, uint64_t out_stride_words, pa_stream_t stream, float *margin) {
    if (n == 0 || m == 0 || m > n || !seed_dev || !keys_dev || !out_dev) return PA_EINVAL;
    if (nkeys < 1 || nkeys > 2) return PA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(seed_dev) | reinterpret_cast<uintptr_t>(keys_dev) |
         reinterpret_cast<uintptr_t>(out_dev)) & 15u)
        return PA_EINVAL;
    if (key_stride_words < (n + 63) / 64 || out_stride_words < (m + 63) / 64) return PA_EINVAL;
    if (nkeys == 2 && ((key_stride_words | out_stride_words) & 1)) return PA_EINVAL;
    if (dtype != PA_FP32_GUARD && dtype != PA_FP64 && dtype != PA_NTT64) return PA_EINVAL;
    int lgL = 12;
    while ((1ull << lgL) < n + m - 1) ++lgL;
    if (lgL > kMaxLgL) return PA_EUNSUPPORTED;  // beyond the static scratch: n + m - 1 must be <= 2^21

    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != PA_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint32_t *marg = reinterpret_cast<uint32_t *>(base + 2 * kSlotBytes + (512u << 10)) + 2;

    if (dtype == PA_NTT64) {
        rc = run_static<Zp>(base, lgL, n, m, seed_dev, keys_dev, nkeys, key_stride_words, out_dev,
                            out_stride_words, st);
        if (rc == PA_OK && margin) margin[0] = 0.f;
        return rc;
    }
    const float guard = static_guard();
    pa_dtype_t mode = dtype;
    for (;;) {
        rc = (mode == PA_FP32_GUARD) ? run_static<float>(base, lgL, n, m, seed_dev, keys_dev, nkeys, key_stride_words,
                                                        out_dev, out_stride_words, st)
                                     : run_static<double>(base, lgL, n, m, seed_dev, keys_dev, nkeys,
                                                          key_stride_words, out_dev, out_stride_words, st);
        if (rc != PA_OK) return rc;
        if (mode == PA_FP64 && !margin) return PA_OK;  // FP64 needs no readback unless asked
        uint32_t mb[2] = {0u, 0u};  // caller's stack, pageable: no allocation
        STATIC_CUDA(cudaMemcpyAsync(mb, marg, nkeys * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        STATIC_CUDA(cudaStreamSynchronize(st));
        float worst = 0.f;
        for (uint32_t k = 0; k < nkeys; ++k) {
            float f;
            memcpy(&f, &mb[k], sizeof(f));
            if (f > worst) worst = f;
        }
        if (worst <= guard) {
            if (margin) margin[0] = worst;
            return PA_OK;
        }
        if (mode == PA_FP64) {  // FP64 failed its guard: recompute exactly
            rc = run_static<Zp>(base, lgL, n, m, seed_dev, keys_dev, nkeys, key_stride_words, out_dev,
                                out_stride_words, st);
            if (rc == PA_OK && margin) margin[0] = 0.f;
            return rc;
        }
        mode = PA_FP64;  // FP32 failed its guard: recompute in FP64 in the same scratch
    }
}

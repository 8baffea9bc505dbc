// pa_api.cu -- the C ABI declared in include/pa.h: plans, seed spectra, batched hashing.
//
// A plan fixes (n, m, dtype) and the transform: complex length L, the smallest
// smooth length ro * 2^k >= n+m-1 (paper Section 2.2: the FFT length of the
// standard Toeplitz hash is n+r-1), split into two or three passes (paper
// Algorithm 1 splits a long FFT into short row and column FFTs with a twiddle
// step in between), the split chosen by timing every candidate. Key pairs share
// one complex transform; a lone key uses a half-length one (RealMode).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pa.h"
#include "pa_launch.h"
#include "pa_internal.h"

using namespace pa;

namespace {
thread_local std::string g_last_cuda_error;
}

// Shared with the other translation units of the library (not part of the C ABI).
int pa_internal_cuda_fail(cudaError_t e, const char *what) {
    g_last_cuda_error = std::string(what) + ": " + cudaGetErrorString(e);
    return PA_ECUDA;
}

namespace {

int cuda_fail(cudaError_t e, const char *what) { return pa_internal_cuda_fail(e, what); }

#define PA_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// Single keys in a half-length transform (FP32 / FP64): one key of a length-2N
// convolution as z[t] = x[2t] + i x[2t+1], split per bin pair (k, N-k) against
// per-bin seed tables, so a lone key costs half the transform work of a key pair.
struct RealMode {
    Geometry geo;  // the length-N transform, N = geo.L
    void *tw_hi = nullptr, *tw_lo = nullptr, *tw_fine = nullptr;
    uint32_t twB = 0;
    void *tabs = nullptr;  // 3N values: E_s, O_s, w_N^k O_s (times 1/N), digit-reversed bin order
    bool seeded = false;
};

// The arguments of an issued batch, kept for its guard step.
struct PendingBatch {
    bool active = false;
    const uint64_t *keys = nullptr;  // device rows the kernels read
    uint32_t nkeys = 0;
    uint64_t kstride = 0;
    uint64_t *out = nullptr;  // device rows the kernels write
    uint64_t ostride = 0;
    pa_stream_t stream = nullptr;
    uint64_t *host_out = nullptr;  // host batches: where the final keys go
    uint64_t host_ostride = 0;
};

struct pa_plan {
    uint64_t n = 0, m = 0;   // the Toeplitz block: m outputs from n transform inputs
    uint64_t n_key = 0;      // key length in bits (n, or n + m for the modified hash)
    uint64_t koff = 0;       // first key bit of the Toeplitz block's input (0, or m)
    bool modified = false;   // modified Toeplitz hash [I_m, T] (Section 2.2, Eq. 2-3)
    pa_dtype_t dtype = PA_FP64;
    int device = 0;
    uint64_t L = 0;
    Geometry geo;  // pass split of L
    uint32_t twB = 0;
    void *tw_hi = nullptr, *tw_lo = nullptr;
    void *tw_fine = nullptr;  // stage twiddles w_F^j, F = geo.F()
    void *spec = nullptr;        // L complex values, seed spectrum in digit-reversed order, times 1/L
    void *work = nullptr;        // work_pairs * L complex values
    uint32_t work_pairs = 0;
    uint32_t max_chunk_pairs = 1;
    uint32_t *popc = nullptr;    // per key
    uint32_t *marg = nullptr;    // per key, float bits
    uint32_t *err = nullptr;     // device words: [0] error bits (bit 0: a bounded copy wait ran out of
                                 // time), [1] and [2] the staged inverse pass's tile ticket and exit count
    bool staged = false;           // last pass as the TMA-staged persistent kernel (pa_plan_set_staged)
    uint32_t store_bits = 0;       // storage-precision study: significand bits kept between passes (0: all)
    uint32_t expire_launches = 0;  // test hook: staged launches left whose first wait is made to run out
    uint32_t key_cap = 0;
    float *h_marg = nullptr;     // pinned: h_cap margins, then the error word
    uint32_t h_cap = 0;
    uint64_t *seed_copy = nullptr;  // the seed bits, kept for an escalation plan
    bool seeded = false;
    float guard = 0.25f;
    pa_plan_t *fallback = nullptr;    // next-wider plan (FP32 -> FP64 -> NTT64) for keys that fail the guard
    RealMode *real = nullptr;         // half-length form for single keys (not in the exact mode)
    PendingBatch pending;             // a batch issued by pa_hash_batch_async, not yet finished
    cudaEvent_t done = nullptr;       // recorded behind the margins' (and host outputs') read-back
    // host batches (pa_hash_host_async): device staging rows and the copy streams around the compute
    uint64_t *stage_keys = nullptr, *stage_out = nullptr;
    size_t stage_key_words = 0, stage_out_words = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in = nullptr, ev_comp = nullptr;
    std::mutex mu;
    // kernel timing
    bool prof = false;
    std::vector<cudaEvent_t> ev_a, ev_b;  // event pairs, reused
    std::vector<int> ev_kind;             // kind of each recorded pair (pending)
    size_t ev_used = 0;
    uint64_t launches[PA_NUM_KERNEL_KINDS] = {};
    double total_ms[PA_NUM_KERNEL_KINDS] = {};
};

namespace {

enum Kind { K_PREP = 0, K_FWD_KEYS, K_FWD_SEED, K_MID_FWD, K_MIDDLE_CONV, K_MIDDLE_SPEC, K_MID_INV, K_INV_BITS };
const char *kKindNames[PA_NUM_KERNEL_KINDS] = {"prep",        "fwd_keys",    "fwd_seed", "mid_fwd",
                                               "middle_conv", "middle_spec", "mid_inv",  "inv_bits"};

// Brackets one launch with a pair of events when timing is on.
struct Timed {
    pa_plan_t *p;
    int kind;
    cudaStream_t st;
    size_t slot = (size_t)-1;
    Timed(pa_plan_t *p_, int kind_, cudaStream_t st_) : p(p_), kind(kind_), st(st_) {
        if (!p->prof) return;
        if (p->ev_used == p->ev_a.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess) return;
            if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
            p->ev_a.push_back(a);
            p->ev_b.push_back(b);
            p->ev_kind.push_back(0);
        }
        slot = p->ev_used++;
        p->ev_kind[slot] = kind;
        cudaEventRecord(p->ev_a[slot], st);
    }
    ~Timed() {
        if (slot != (size_t)-1) cudaEventRecord(p->ev_b[slot], st);
    }
};

void collect_events(pa_plan_t *p) {
    for (size_t i = 0; i < p->ev_used; ++i) {
        float ms = 0.f;
        if (cudaEventSynchronize(p->ev_b[i]) == cudaSuccess && cudaEventElapsedTime(&ms, p->ev_a[i], p->ev_b[i]) == cudaSuccess) {
            p->total_ms[p->ev_kind[i]] += ms;
            p->launches[p->ev_kind[i]] += 1;
        }
    }
    p->ev_used = 0;
}

size_t elem_bytes(pa_dtype_t d) {
    return d == PA_FP32_GUARD ? sizeof(float2) : d == PA_FP64 ? sizeof(double2) : sizeof(uint64_t);
}

// ---- modular helpers (host) for the NTT mode -------------------------------------------------
uint64_t zp_mul_host(uint64_t a, uint64_t b) {
    unsigned __int128 x = (unsigned __int128)a * b;
    return zp_reduce((uint64_t)(x >> 64), (uint64_t)x);
}
uint64_t zp_pow_host(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = zp_mul_host(r, a);
        a = zp_mul_host(a, a);
        e >>= 1;
    }
    return r;
}
// Root of unity of order L (a power of two, 32 <= L <= 2^32) whose L/32-th power
// is 2^6, the root the in-register DFTs use.
uint64_t zp_root(uint64_t L) {
    const uint64_t g = 7;  // generates the multiplicative group mod p
    const uint64_t w = zp_pow_host(g, (kP - 1) / L);
    const uint64_t w32 = zp_pow_host(w, L / 32);
    for (uint64_t j = 1; j < 64; j += 2) {
        if (zp_pow_host(w32, j) == 64ull) return zp_pow_host(w, j);
    }
    return 0;
}

template <typename T>
int make_twiddles(uint64_t Lu, uint32_t F, void **dhi, void **dlo, uint32_t *Bout, void **dfine) {
    int lgL = 0;
    while ((1ull << lgL) < Lu) ++lgL;
    const uint32_t B = (uint32_t)(lgL + 1) / 2;
    const uint64_t nlo = 1ull << B, nhi = (Lu + nlo - 1) >> B;
    std::vector<cx<T>> hi(nhi), lo(nlo), fine(F);
    const double L = (double)Lu;
    const double two_pi = 6.283185307179586476925286766559;
    for (uint64_t h = 0; h < nhi; ++h) {
        const double a = two_pi * (double)(h << B) / L;
        hi[h].x = (T)std::cos(a);
        hi[h].y = (T)-std::sin(a);
    }
    for (uint64_t l = 0; l < nlo; ++l) {
        const double a = two_pi * (double)l / L;
        lo[l].x = (T)std::cos(a);
        lo[l].y = (T)-std::sin(a);
    }
    for (uint64_t j = 0; j < F; ++j) {
        const double a = two_pi * (double)j / (double)F;
        fine[j].x = (T)std::cos(a);
        fine[j].y = (T)-std::sin(a);
    }
    PA_CUDA(cudaMalloc(dhi, nhi * sizeof(cx<T>)));
    PA_CUDA(cudaMalloc(dlo, nlo * sizeof(cx<T>)));
    PA_CUDA(cudaMalloc(dfine, (size_t)F * sizeof(cx<T>)));
    PA_CUDA(cudaMemcpy(*dhi, hi.data(), nhi * sizeof(cx<T>), cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(*dlo, lo.data(), nlo * sizeof(cx<T>), cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(*dfine, fine.data(), (size_t)F * sizeof(cx<T>), cudaMemcpyHostToDevice));
    *Bout = B;
    return PA_OK;
}

template <>
int make_twiddles<Zp>(uint64_t Lu, uint32_t F, void **dhi, void **dlo, uint32_t *Bout, void **dfine) {
    if (Lu & (Lu - 1)) return PA_EUNSUPPORTED;  // the exact transform keeps power-of-two lengths
    int lgL = 0;
    while ((1ull << lgL) < Lu) ++lgL;
    const uint32_t B = (uint32_t)(lgL + 1) / 2;
    const uint64_t nhi = 1ull << (lgL - B), nlo = 1ull << B;
    std::vector<uint64_t> hi(nhi), lo(nlo), fine(F);
    const uint64_t w = zp_root(Lu);
    if (w == 0 || Lu % F) return PA_EUNSUPPORTED;
    const uint64_t wB = zp_pow_host(w, 1ull << B);
    uint64_t x = 1;
    for (uint64_t h = 0; h < nhi; ++h) { hi[h] = x; x = zp_mul_host(x, wB); }
    x = 1;
    for (uint64_t l = 0; l < nlo; ++l) { lo[l] = x; x = zp_mul_host(x, w); }
    const uint64_t wF = zp_pow_host(w, Lu / F);  // w_F = w_L^(L/F): the same root system
    x = 1;
    for (uint64_t j = 0; j < F; ++j) { fine[j] = x; x = zp_mul_host(x, wF); }
    PA_CUDA(cudaMalloc(dhi, nhi * sizeof(uint64_t)));
    PA_CUDA(cudaMalloc(dlo, nlo * sizeof(uint64_t)));
    PA_CUDA(cudaMalloc(dfine, (size_t)F * sizeof(uint64_t)));
    PA_CUDA(cudaMemcpy(*dhi, hi.data(), nhi * sizeof(uint64_t), cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(*dlo, lo.data(), nlo * sizeof(uint64_t), cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(*dfine, fine.data(), (size_t)F * sizeof(uint64_t), cudaMemcpyHostToDevice));
    *Bout = B;
    return PA_OK;
}

template <typename T>
int build_twiddles(pa_plan_t *p) {
    return make_twiddles<T>(p->L, p->geo.F(), &p->tw_hi, &p->tw_lo, &p->twB, &p->tw_fine);
}

// 1/L as the element type's scaling factor.
template <typename T> cx<T> inv_length(uint64_t L) {
    cx<T> s;
    s.x = (decltype(s.x))(1.0 / (double)L);
    s.y = 0;
    return s;
}
template <> cx<Zp> inv_length<Zp>(uint64_t L) { return zp_pow_host(L, kP - 2); }
template <typename T> cx<T> one() { return inv_length<T>(1); }

template <typename T>
TwTab<T> tw_of(const pa_plan_t *p) {
    TwTab<T> t;
    t.hi = static_cast<const cx<T> *>(p->tw_hi);
    t.lo = static_cast<const cx<T> *>(p->tw_lo);
    t.B = p->twB;
    t.lgL = 0;
    while ((1ull << t.lgL) < p->L) ++t.lgL;  // log2 L for the power-of-two lengths of the exact transform
    t.fine = static_cast<const cx<T> *>(p->tw_fine);
    t.F = p->geo.F();
    return t;
}

template <typename T>
TwTab<T> tw_of_real(const RealMode *r) {
    TwTab<T> t;
    t.hi = static_cast<const cx<T> *>(r->tw_hi);
    t.lo = static_cast<const cx<T> *>(r->tw_lo);
    t.B = r->twB;
    t.lgL = 0;
    while ((1ull << t.lgL) < r->geo.L) ++t.lgL;
    t.fine = static_cast<const cx<T> *>(r->tw_fine);
    t.F = r->geo.F();
    return t;
}

int ensure_work(pa_plan_t *p, uint32_t pairs) {
    if (pairs <= p->work_pairs) return PA_OK;
    if (p->work) {
        cudaError_t e = cudaFree(p->work);
        p->work = nullptr;
        p->work_pairs = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(work)");
    }
    cudaError_t e = cudaMalloc(&p->work, (size_t)pairs * p->L * elem_bytes(p->dtype));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return PA_ENOMEM;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(work)");
    p->work_pairs = pairs;
    return PA_OK;
}

int ensure_keys(pa_plan_t *p, uint32_t nkeys) {
    if (nkeys <= p->key_cap) return PA_OK;
    if (p->popc) cudaFree(p->popc);
    if (p->marg) cudaFree(p->marg);
    p->popc = p->marg = nullptr;
    p->key_cap = 0;
    PA_CUDA(cudaMalloc(&p->popc, (size_t)nkeys * sizeof(uint32_t)));
    PA_CUDA(cudaMalloc(&p->marg, (size_t)nkeys * sizeof(uint32_t)));
    p->key_cap = nkeys;
    return PA_OK;
}

int ensure_host(pa_plan_t *p, uint32_t nkeys) {
    if (nkeys <= p->h_cap) return PA_OK;
    if (p->h_marg) cudaFreeHost(p->h_marg);
    p->h_marg = nullptr;
    p->h_cap = 0;
    PA_CUDA(cudaMallocHost(&p->h_marg, ((size_t)nkeys + 1) * sizeof(float)));
    p->h_cap = nkeys;
    return PA_OK;
}

// Pairs per launch chunk: bounded by the work-buffer budget and by the grid's
// y extent (65535) of the three-level middle strided pass.
uint32_t chunk_pairs_limit(const pa_plan_t *p) {
    size_t budget = (size_t)4 << 30;  // 4 GiB of work buffer
    if (const char *s = std::getenv("PA_WORK_BYTES")) budget = (size_t)std::strtoull(s, nullptr, 10);
    size_t per = (size_t)p->L * elem_bytes(p->dtype);
    size_t lim = budget / per;
    if (lim < 1) lim = 1;
    if (p->geo.lgM) {
        size_t nblk = (size_t)1 << p->geo.lg1;
        size_t y = 65535 / nblk;
        if (y < lim) lim = y;
    }
    if (lim > 65535) lim = 65535;
    return (uint32_t)lim;
}

// Storage-precision study (pa_plan_set_storage_bits): round `pairs` slots of values a pass
// has just stored to the plan's significand width. Only FP32 plans carry the setting.
template <typename T>
cudaError_t round_stored(const pa_plan_t *p, cx<T> *slots, uint32_t pairs, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (p->store_bits) return launch_round_significand(reinterpret_cast<float *>(slots), 2ull * pairs * p->L, p->store_bits, st);
    }
    return cudaSuccess;
}

template <typename T>
int run_seed(pa_plan_t *p, const uint64_t *seed, cudaStream_t st) {
    const TwTab<T> tw = tw_of<T>(p);
    cx<T> *W = static_cast<cx<T> *>(p->work);
    cx<T> *spec = static_cast<cx<T> *>(p->spec);
    const Geometry &g = p->geo;
    { Timed t_(p, K_FWD_SEED, st); PA_CUDA(launch_fwd_seed<T>(g.lg1, seed, p->n, p->m, W, p->L, tw, st)); }
    if (g.lgM) {
        Timed t_(p, K_MID_FWD, st);
        PA_CUDA(launch_mid<T>(g.lgM, false, W, p->L, g.inner(), 1, tw, st));
    }
    { Timed t_(p, K_MIDDLE_SPEC, st); PA_CUDA(launch_middle<T>(g.ro, g.lgI, 1, W, spec, p->L, 1, tw, inv_length<T>(p->L), st)); }
    PA_CUDA(round_stored<T>(p, spec, 1, st));
    return PA_OK;
}

// Seed tables of the half-length form: packed seed transform, then the bin-pair split.
template <typename T>
int run_seed_real(pa_plan_t *p, const uint64_t *seed, cudaStream_t st) {
    RealMode *r = p->real;
    const TwTab<T> tw = tw_of_real<T>(r);
    cx<T> *W = static_cast<cx<T> *>(p->work);
    const Geometry &g = r->geo;
    const uint64_t N = g.L;
    PA_CUDA(launch_fwd_seed<T>(g.lg1, seed, p->n, p->m, W, N, tw, st, true));
    if (g.lgM) PA_CUDA(launch_mid<T>(g.lgM, false, W, N, g.inner(), 1, tw, st));
    PA_CUDA(launch_middle_real<T>(g.ro, g.lgI, 1, W, static_cast<cx<T> *>(r->tabs), N, (uint32_t)g.lg1,
                                  (uint32_t)g.lgM, tw, (T)(1.0 / (double)N), 1, st));
    return PA_OK;
}

// Keys through the half-length form, one key per slot of N values (as many slots per
// launch as the work buffer holds).
template <typename T>
int run_keys_real(pa_plan_t *p, const uint64_t *keys, uint32_t nkeys, uint64_t kstride, uint64_t *out,
                  uint64_t ostride, uint32_t *popc, uint32_t *marg, cudaStream_t st) {
    RealMode *r = p->real;
    const TwTab<T> tw = tw_of_real<T>(r);
    cx<T> *W = static_cast<cx<T> *>(p->work);
    cx<T> *tabs = static_cast<cx<T> *>(r->tabs);
    const Geometry &g = r->geo;
    const uint64_t N = g.L;
    uint64_t cap = (uint64_t)p->work_pairs * p->L / N;  // slots that fit the work buffer
    if (cap < 1) cap = 1;
    if (g.lgM && cap > 65535u >> g.lg1) cap = 65535u >> g.lg1;  // grid y of the middle strided pass
    { Timed t_(p, K_PREP, st); PA_CUDA(launch_zero_keys(nkeys, popc, marg, st)); }
    for (uint32_t k0 = 0; k0 < nkeys; k0 += (uint32_t)cap) {
        const uint32_t ns = (nkeys - k0 < cap) ? nkeys - k0 : (uint32_t)cap;
        const uint64_t *kp = keys + (uint64_t)k0 * kstride;
        uint64_t *op = out + (uint64_t)k0 * ostride;
        { Timed t_(p, K_FWD_KEYS, st); PA_CUDA(launch_fwd_keys<T>(g.lg1, kp, ns, kstride, p->n, W, N, ns, tw, popc + k0, st, p->koff, true)); }
        if (g.lgM) { Timed t_(p, K_MID_FWD, st); PA_CUDA(launch_mid<T>(g.lgM, false, W, N, g.inner(), ns, tw, st)); }
        { Timed t_(p, K_MIDDLE_CONV, st); PA_CUDA(launch_middle_real<T>(g.ro, g.lgI, 0, W, tabs, N, (uint32_t)g.lg1, (uint32_t)g.lgM, tw, (T)1, ns, st)); }
        if (g.lgM) { Timed t_(p, K_MID_INV, st); PA_CUDA(launch_mid<T>(g.lgM, true, W, N, g.inner(), ns, tw, st)); }
        { Timed t_(p, K_INV_BITS, st); PA_CUDA(launch_inv_bits<T>(g.lg1, W, N, p->m, ns, popc + k0, marg + k0, op, ostride, ns, tw, st, p->modified ? kp : nullptr, kstride, true)); }
    }
    return PA_OK;
}

// Wait limit handed to the next launch of the TMA-staged inverse pass: 0 (the kernel's
// own 1 s limit, copies issued as usual), or, while the test hook of
// pa_plan_expire_waits is armed, 10 us on a barrier phase that no copy completes.
uint32_t take_expire(pa_plan_t *p) {
    if (p->expire_launches == 0) return 0u;
    --p->expire_launches;
    return 10000u;
}

template <typename T>
int run_keys(pa_plan_t *p, const uint64_t *keys, uint32_t nkeys, uint64_t kstride, uint64_t *out,
             uint64_t ostride, uint32_t *popc, uint32_t *marg, cudaStream_t st) {
    if constexpr (!std::is_same<T, Zp>::value) {
        // A lone key (alone, or the last of an odd batch) takes the half-length form; key
        // pairs stay in the pair form (measured 28 % faster per key than the half-length form).
        if (p->real && p->real->seeded && (nkeys & 1) && p->store_bits == 0) {
            if (nkeys > 1) {
                const int rc = run_keys<T>(p, keys, nkeys - 1, kstride, out, ostride, popc, marg, st);
                if (rc != PA_OK) return rc;
            }
            const uint32_t k = nkeys - 1;
            return run_keys_real<T>(p, keys + (uint64_t)k * kstride, 1, kstride, out + (uint64_t)k * ostride,
                                    ostride, popc + k, marg + k, st);
        }
    }
    const TwTab<T> tw = tw_of<T>(p);
    cx<T> *W = static_cast<cx<T> *>(p->work);
    cx<T> *spec = static_cast<cx<T> *>(p->spec);
    const Geometry &g = p->geo;
    { Timed t_(p, K_PREP, st); PA_CUDA(launch_zero_keys(nkeys, popc, marg, st)); }
    const uint32_t npairs = (nkeys + 1) / 2;
    for (uint32_t p0 = 0; p0 < npairs; p0 += p->work_pairs) {
        const uint32_t pairs = (npairs - p0 < p->work_pairs) ? npairs - p0 : p->work_pairs;
        const uint32_t k0 = 2 * p0;
        const uint32_t nk = (nkeys - k0 < 2 * pairs) ? nkeys - k0 : 2 * pairs;
        const uint64_t *kp = keys + (uint64_t)k0 * kstride;
        uint64_t *op = out + (uint64_t)k0 * ostride;
        { Timed t_(p, K_FWD_KEYS, st); PA_CUDA(launch_fwd_keys<T>(g.lg1, kp, nk, kstride, p->n, W, p->L, pairs, tw, popc + k0, st, p->koff)); }
        PA_CUDA(round_stored<T>(p, W, pairs, st));
        if (g.lgM) {
            { Timed t_(p, K_MID_FWD, st); PA_CUDA(launch_mid<T>(g.lgM, false, W, p->L, g.inner(), pairs, tw, st)); }
            PA_CUDA(round_stored<T>(p, W, pairs, st));
            { Timed t_(p, K_MIDDLE_CONV, st); PA_CUDA(launch_middle<T>(g.ro, g.lgI, 0, W, spec, p->L, pairs, tw, one<T>(), st)); }
            PA_CUDA(round_stored<T>(p, W, pairs, st));
            { Timed t_(p, K_MID_INV, st); PA_CUDA(launch_mid<T>(g.lgM, true, W, p->L, g.inner(), pairs, tw, st)); }
        } else {
            Timed t_(p, K_MIDDLE_CONV, st);
            PA_CUDA(launch_middle<T>(g.ro, g.lgI, 0, W, spec, p->L, pairs, tw, one<T>(), st));
        }
        PA_CUDA(round_stored<T>(p, W, pairs, st));
        { Timed t_(p, K_INV_BITS, st); PA_CUDA(launch_inv_bits<T>(g.lg1, W, p->L, p->m, nk, popc + k0, marg + k0, op, ostride, pairs, tw, st, p->modified ? kp : nullptr, kstride, false, p->staged ? p->err : nullptr, take_expire(p))); }
    }
    return PA_OK;
}

void free_real_mode(pa_plan_t *p) {
    if (!p->real) return;
    cudaFree(p->real->tw_hi);
    cudaFree(p->real->tw_lo);
    cudaFree(p->real->tw_fine);
    cudaFree(p->real->tabs);
    delete p->real;
    p->real = nullptr;
}

void free_plan(pa_plan_t *p) {
    if (!p) return;
    if (p->fallback) free_plan(p->fallback);
    cudaFree(p->tw_hi);
    cudaFree(p->tw_lo);
    cudaFree(p->tw_fine);
    cudaFree(p->spec);
    cudaFree(p->work);
    cudaFree(p->popc);
    cudaFree(p->marg);
    cudaFree(p->err);
    cudaFree(p->seed_copy);
    if (p->h_marg) cudaFreeHost(p->h_marg);
    if (p->done) cudaEventDestroy(p->done);
    free_real_mode(p);
    cudaFree(p->stage_keys);
    cudaFree(p->stage_out);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_comp) cudaEventDestroy(p->ev_comp);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    for (cudaEvent_t e : p->ev_a) cudaEventDestroy(e);
    for (cudaEvent_t e : p->ev_b) cudaEventDestroy(e);
    delete p;
}

bool plan_args_ok(uint64_t n, uint64_t m, pa_dtype_t dtype) {
    if (n == 0 || m == 0 || m > n || n > (1ull << 27)) return false;
    return dtype == PA_FP64 || dtype == PA_FP32_GUARD || dtype == PA_NTT64;
}

// Modified hash: key of n bits, identity block m x m, Toeplitz block m x (n - m); 1 <= m < n.
bool modified_args_ok(uint64_t n, uint64_t m, pa_dtype_t dtype) {
    if (m == 0 || m >= n || n > (1ull << 27)) return false;
    return dtype == PA_FP64 || dtype == PA_FP32_GUARD || dtype == PA_NTT64;
}

// Pass lengths of a split as the ABI reports them: L1, then the middle strided pass
// and the innermost pass for three passes, else the innermost pass and 1.
void split_lengths(const Geometry &g, uint32_t *L1, uint32_t *L2, uint32_t *L3) {
    *L1 = 1u << g.lg1;
    *L2 = g.lgM ? (1u << g.lgM) : g.inner();
    *L3 = g.lgM ? g.inner() : 1u;
}

int build_plan_twiddles(pa_plan_t *p) {
    return (p->dtype == PA_FP32_GUARD) ? build_twiddles<float>(p)
           : (p->dtype == PA_FP64)     ? build_twiddles<double>(p)
                                       : build_twiddles<Zp>(p);
}

void free_plan_twiddles(pa_plan_t *p) {
    cudaFree(p->tw_hi);
    cudaFree(p->tw_lo);
    cudaFree(p->tw_fine);
    p->tw_hi = p->tw_lo = p->tw_fine = nullptr;
}

// ---- split autotuner ---------------------------------------------------------------------------
// Every valid split of a transform length runs the same arithmetic in a different
// pass structure; which one is fastest depends on the kernel instances and is
// measured, not modelled: once per (L, dtype) and process, each candidate hashes a
// batch of all-zero keys (the kernels' cost does not depend on the bit values)
// and the fastest is kept. PA_PLAN_TUNE=0 turns it off (the default split is used).
std::mutex g_split_mu;
std::map<std::pair<uint64_t, int>, Geometry> g_split;

bool tuning_enabled() {
    const char *s = std::getenv("PA_PLAN_TUNE");
    return !(s && s[0] == '0');
}

// Median of five timed runs after one warm-up run (which also loads the kernels).
template <typename T>
int time_split(pa_plan_t *p, uint32_t nkeys, const uint64_t *keys, uint64_t kw, uint64_t *out, uint64_t ow,
               cudaStream_t st, cudaEvent_t a, cudaEvent_t b, float *ms) {
    float t[6] = {};
    for (int rep = 0; rep < 6; ++rep) {
        PA_CUDA(cudaEventRecord(a, st));
        int rc = run_keys<T>(p, keys, nkeys, kw, out, ow, p->popc, p->marg, st);
        if (rc != PA_OK) return rc;
        PA_CUDA(cudaEventRecord(b, st));
        PA_CUDA(cudaEventSynchronize(b));
        PA_CUDA(cudaEventElapsedTime(&t[rep], a, b));
    }
    std::sort(t + 1, t + 6);
    *ms = t[3];
    return PA_OK;
}

// Chooses p->geo among the candidates of p->L (cached per process). The plan's spectrum
// slot must exist; twiddles and work buffers made for the trials are released again.
int tune_split(pa_plan_t *p, const std::vector<Geometry> &cand) {
    const std::pair<uint64_t, int> key{p->L, (int)p->dtype};
    {
        std::lock_guard<std::mutex> lk(g_split_mu);
        auto it = g_split.find(key);
        if (it != g_split.end()) {
            p->geo = it->second;
            return PA_OK;
        }
    }
    const size_t per_pair = (size_t)p->L * elem_bytes(p->dtype);
    uint32_t pairs = (uint32_t)(((size_t)512 << 20) / per_pair);  // about 512 MB of work: well past the L2
    if (pairs < 1) pairs = 1;
    if (pairs > 32) pairs = 32;
    if (pairs > p->max_chunk_pairs) pairs = p->max_chunk_pairs;
    const uint32_t nkeys = 2 * pairs;
    const uint64_t kw = ((p->n_key + 63) / 64 + 1) & ~1ull, ow = ((p->m + 63) / 64 + 1) & ~1ull;
    uint64_t *keys = nullptr, *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = PA_OK;
    float best = 0.f;
    Geometry bestg = p->geo;
    auto fail = [&](int r) {
        cudaFree(keys);
        cudaFree(out);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (st) cudaStreamDestroy(st);
        return r;
    };
    cudaError_t e = cudaMalloc(&keys, (size_t)nkeys * kw * 8);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)nkeys * ow * 8);
    if (e == cudaSuccess) e = cudaMemset(keys, 0, (size_t)nkeys * kw * 8);
    if (e == cudaSuccess) e = cudaMemset(p->spec, 0, per_pair);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(PA_ENOMEM);
    }
    if (e != cudaSuccess) return fail(cuda_fail(e, "split autotuner set-up"));
    if ((rc = ensure_work(p, pairs)) != PA_OK || (rc = ensure_keys(p, nkeys)) != PA_OK) return fail(rc);
    for (size_t i = 0; i < cand.size(); ++i) {
        p->geo = cand[i];
        if ((rc = build_plan_twiddles(p)) != PA_OK) return fail(rc);
        float ms = 0.f;
        rc = (p->dtype == PA_FP32_GUARD) ? time_split<float>(p, nkeys, keys, kw, out, ow, st, a, b, &ms)
             : (p->dtype == PA_FP64)     ? time_split<double>(p, nkeys, keys, kw, out, ow, st, a, b, &ms)
                                         : time_split<Zp>(p, nkeys, keys, kw, out, ow, st, a, b, &ms);
        free_plan_twiddles(p);
        if (rc != PA_OK) return fail(rc);
        if (i == 0 || ms < best) {
            best = ms;
            bestg = cand[i];
        }
    }
    p->geo = bestg;
    // The trial work buffer is sized for the trials, not for this plan's batches.
    cudaFree(p->work);
    p->work = nullptr;
    p->work_pairs = 0;
    {
        std::lock_guard<std::mutex> lk(g_split_mu);
        g_split[key] = bestg;
    }
    return fail(PA_OK);
}

// The half-length form of a plan: the smallest supported N with 2N >= n+m-1 whose
// innermost pass fits the two-row kernel; left out (nullptr) if there is none.
// Split autotuner of the half-length form (as tune_split, on one zero key, cached per
// (N, dtype)). r->tabs must exist; the chosen split's twiddles are built by the caller.
std::map<std::pair<uint64_t, int>, Geometry> g_real_split;

template <typename T>
int time_real(pa_plan_t *p, const uint64_t *key, uint64_t kw, uint64_t *out, uint64_t ow, cudaStream_t st,
              cudaEvent_t a, cudaEvent_t b, float *ms) {
    float t[6] = {};
    for (int rep = 0; rep < 6; ++rep) {
        PA_CUDA(cudaEventRecord(a, st));
        int rc = run_keys_real<T>(p, key, 1, kw, out, ow, p->popc, p->marg, st);
        if (rc != PA_OK) return rc;
        PA_CUDA(cudaEventRecord(b, st));
        PA_CUDA(cudaEventSynchronize(b));
        PA_CUDA(cudaEventElapsedTime(&t[rep], a, b));
    }
    std::sort(t + 1, t + 6);
    *ms = t[3];
    return PA_OK;
}

int tune_real(pa_plan_t *p, RealMode *r) {
    const std::pair<uint64_t, int> cache_key{r->geo.L, (int)p->dtype};
    {
        std::lock_guard<std::mutex> lk(g_split_mu);
        auto it = g_real_split.find(cache_key);
        if (it != g_real_split.end()) {
            r->geo = it->second;
            return PA_OK;
        }
    }
    const std::vector<Geometry> cand = geometry_candidates(r->geo.L, p->dtype, true);
    if (cand.size() < 2 || !tuning_enabled()) return PA_OK;
    const uint64_t kw = (p->n_key + 63) / 64, ow = (p->m + 63) / 64;
    uint64_t *key = nullptr, *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    auto done = [&](int rc) {
        cudaFree(key);
        cudaFree(out);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (st) cudaStreamDestroy(st);
        return rc;
    };
    cudaError_t e = cudaMalloc(&key, kw * 8);
    if (e == cudaSuccess) e = cudaMalloc(&out, ow * 8);
    if (e == cudaSuccess) e = cudaMemset(key, 0, kw * 8);
    if (e == cudaSuccess) e = cudaMemset(r->tabs, 0, (size_t)3 * r->geo.L * elem_bytes(p->dtype));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return done(PA_ENOMEM);
    }
    if (e != cudaSuccess) return done(cuda_fail(e, "half-length autotuner set-up"));
    int rc = ensure_work(p, 1);
    if (rc == PA_OK) rc = ensure_keys(p, 1);
    if (rc != PA_OK) return done(rc);
    float best = 0.f;
    Geometry bestg = r->geo;
    for (size_t i = 0; i < cand.size(); ++i) {
        r->geo = cand[i];
        rc = pa_internal_twiddles(r->geo.L, r->geo.F(), (int)p->dtype, &r->tw_hi, &r->tw_lo, &r->twB, &r->tw_fine);
        float ms = 0.f;
        if (rc == PA_OK)
            rc = (p->dtype == PA_FP32_GUARD) ? time_real<float>(p, key, kw, out, ow, st, a, b, &ms)
                                             : time_real<double>(p, key, kw, out, ow, st, a, b, &ms);
        cudaFree(r->tw_hi);
        cudaFree(r->tw_lo);
        cudaFree(r->tw_fine);
        r->tw_hi = r->tw_lo = r->tw_fine = nullptr;
        if (rc != PA_OK) return done(rc);
        if (i == 0 || ms < best) {
            best = ms;
            bestg = cand[i];
        }
    }
    r->geo = bestg;
    {
        std::lock_guard<std::mutex> lk(g_split_mu);
        g_real_split[cache_key] = bestg;
    }
    return done(PA_OK);
}

int build_real_mode(pa_plan_t *p) {
    const uint64_t need = p->n + p->m - 1;
    const Geometry g = choose_geometry((need + 1) / 2, p->dtype, true);
    if (g.L == 0) return PA_OK;
    RealMode *r = new RealMode();
    r->geo = g;
    p->real = r;  // released with the plan, also on failure
    cudaError_t e = cudaMalloc(&r->tabs, (size_t)3 * g.L * elem_bytes(p->dtype));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return PA_ENOMEM;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(real tables)");
    int rc = tune_real(p, r);
    if (rc != PA_OK) return rc;
    return pa_internal_twiddles(r->geo.L, r->geo.F(), (int)p->dtype, &r->tw_hi, &r->tw_lo, &r->twB, &r->tw_fine);
}

// pa_plan (or pa_plan_modified), with the split forced when `force` is given. For the
// modified hash, n is the key length and the Toeplitz block is m x (n - m).
int plan_create(uint64_t n, uint64_t m, pa_dtype_t dtype, const Geometry *force, pa_plan_t **out,
                bool modified = false) {
    if (!out) return PA_EINVAL;
    *out = nullptr;
    if (modified ? !modified_args_ok(n, m, dtype) : !plan_args_ok(n, m, dtype)) return PA_EINVAL;
    pa_plan_t *p = new pa_plan_t();
    p->modified = modified;
    p->n_key = n;
    p->koff = modified ? m : 0;
    p->n = modified ? n - m : n;
    p->m = m;
    p->dtype = dtype;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    }
    const Geometry geo = force ? *force : choose_geometry(p->n + m - 1, dtype, false);
    if (geo.L == 0) {
        delete p;
        return PA_EUNSUPPORTED;
    }
    p->L = geo.L;
    p->geo = geo;
    cudaError_t e = cudaMalloc(&p->spec, (size_t)p->L * elem_bytes(dtype));
    if (e == cudaSuccess) e = cudaMalloc(&p->err, 4 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(p->err, 0, 4 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);  // zero before any stream of the plan uses them
    if (e != cudaSuccess) {
        free_plan(p);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return PA_ENOMEM;
        }
        return cuda_fail(e, "cudaMalloc(spec)");
    }
    p->max_chunk_pairs = chunk_pairs_limit(p);
    int rc = PA_OK;
    if (!force && tuning_enabled()) {
        const std::vector<Geometry> cand = geometry_candidates(p->L, dtype, false);
        if (cand.size() > 1) rc = tune_split(p, cand);
    }
    if (rc == PA_OK) rc = build_plan_twiddles(p);
    if (rc == PA_OK && dtype != PA_NTT64 && build_real_mode(p) != PA_OK) {
        // The half-length form is an optimisation: without memory for its tables a lone
        // key takes the pair form instead.
        free_real_mode(p);
        cudaGetLastError();
    }
    if (rc != PA_OK) {
        free_plan(p);
        return rc;
    }
    p->max_chunk_pairs = chunk_pairs_limit(p);  // depends on the split
    *out = p;
    return PA_OK;
}

// Recomputes key k of a finished batch with the plan's fallback (one mode wider), in
// stream order on the batch's stream, and reports the margin and mode that produced it.
int escalate_key(pa_plan_t *p, const PendingBatch &b, uint32_t k, float *margin, int32_t *mode) {
    if (!p->fallback->seeded) {
        int rc = pa_set_seed(p->fallback, p->seed_copy, p->n + p->m - 1, b.stream);
        if (rc != PA_OK) return rc;
    }
    float m2 = 0.f;
    int32_t mode2 = 0;
    pa_batch_info_t sub{&m2, &mode2, 0, 0};
    int rc = pa_hash_batch(p->fallback, b.keys + (uint64_t)k * b.kstride, 1, b.kstride, b.out + (uint64_t)k * b.ostride,
                           b.ostride, b.stream, &sub);
    if (rc != PA_OK) return rc;
    if (b.host_out) {  // the batch's read-back carried the first result: replace this key's row
        cudaStream_t st = reinterpret_cast<cudaStream_t>(b.stream);
        PA_CUDA(cudaMemcpyAsync(b.host_out + (uint64_t)k * b.host_ostride, b.out + (uint64_t)k * b.ostride,
                                (size_t)((p->m + 63) / 64) * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        PA_CUDA(cudaStreamSynchronize(st));
    }
    *margin = m2;
    *mode = mode2;
    return PA_OK;
}

// Kernels of one batch and the read-back of its margins and error word, on st.
int issue_batch(pa_plan_t *p, const uint64_t *keys_dev, uint32_t nkeys, uint64_t kstride, uint64_t *out_dev,
                uint64_t ostride, cudaStream_t st) {
    const uint32_t npairs = (nkeys + 1) / 2;
    uint32_t want = npairs < p->max_chunk_pairs ? npairs : p->max_chunk_pairs;
    int rc = ensure_work(p, want);
    if (rc != PA_OK) return rc;
    rc = ensure_keys(p, nkeys);
    if (rc != PA_OK) return rc;
    rc = ensure_host(p, nkeys);
    if (rc != PA_OK) return rc;
    if (!p->done) PA_CUDA(cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming));
    // The plan's work buffers are shared by its batches: a batch issued on another stream
    // than the previous one waits for it (a no-op on the same stream).
    PA_CUDA(cudaStreamWaitEvent(st, p->done, 0));
    if (p->dtype == PA_FP32_GUARD)
        rc = run_keys<float>(p, keys_dev, nkeys, kstride, out_dev, ostride, p->popc, p->marg, st);
    else if (p->dtype == PA_FP64)
        rc = run_keys<double>(p, keys_dev, nkeys, kstride, out_dev, ostride, p->popc, p->marg, st);
    else
        rc = run_keys<Zp>(p, keys_dev, nkeys, kstride, out_dev, ostride, p->popc, p->marg, st);
    if (rc != PA_OK) return rc;
    // the margins and the error word travel back behind the kernels; pa_batch_finish waits for them
    PA_CUDA(cudaMemcpyAsync(p->h_marg, p->marg, (size_t)nkeys * sizeof(float), cudaMemcpyDeviceToHost, st));
    PA_CUDA(cudaMemcpyAsync(p->h_marg + nkeys, p->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    return PA_OK;
}

int ensure_staging(pa_plan_t *p, size_t key_words, size_t out_words) {
    if (key_words > p->stage_key_words) {
        cudaFree(p->stage_keys);
        p->stage_keys = nullptr;
        p->stage_key_words = 0;
        cudaError_t e = cudaMalloc(&p->stage_keys, key_words * sizeof(uint64_t));
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return PA_ENOMEM;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(stage_keys)");
        p->stage_key_words = key_words;
    }
    if (out_words > p->stage_out_words) {
        cudaFree(p->stage_out);
        p->stage_out = nullptr;
        p->stage_out_words = 0;
        cudaError_t e = cudaMalloc(&p->stage_out, out_words * sizeof(uint64_t));
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return PA_ENOMEM;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(stage_out)");
        p->stage_out_words = out_words;
    }
    if (!p->s_in) PA_CUDA(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking));
    if (!p->s_out) PA_CUDA(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking));
    if (!p->ev_in) PA_CUDA(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
    if (!p->ev_comp) PA_CUDA(cudaEventCreateWithFlags(&p->ev_comp, cudaEventDisableTiming));
    return PA_OK;
}

}  // namespace

int pa_internal_twiddles(uint64_t L, uint32_t F, int dtype, void **hi, void **lo, uint32_t *B, void **fine) {
    return dtype == PA_FP32_GUARD ? make_twiddles<float>(L, F, hi, lo, B, fine)
           : dtype == PA_FP64     ? make_twiddles<double>(L, F, hi, lo, B, fine)
                                  : make_twiddles<Zp>(L, F, hi, lo, B, fine);
}

extern "C" {

const char *pa_strerror(int code) {
    switch (code) {
        case PA_OK: return "PA_OK: success";
        case PA_EINVAL: return "PA_EINVAL: invalid argument (size, pointer, alignment, stride or handle)";
        case PA_ENOMEM: return "PA_ENOMEM: device or pinned host memory exhausted";
        case PA_EAGAIN: return "PA_EAGAIN: admission cap reached and queue full";
        case PA_EPENDING: return "PA_EPENDING: request not complete yet";
        case PA_ETIMEOUT: return "PA_ETIMEOUT: bounded wait expired";
        case PA_EPRECISION: return "PA_EPRECISION: no precision mode rounded unambiguously";
        case PA_ECUDA: return "PA_ECUDA: CUDA runtime error";
        case PA_ENOSEED: return "PA_ENOSEED: pa_set_seed has not been called on this plan";
        case PA_EUNSUPPORTED: return "PA_EUNSUPPORTED: size or mode not supported by this build";
        default: return "unknown pa error code";
    }
}

const char *pa_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int pa_plan(uint64_t n, uint64_t m, pa_dtype_t dtype, pa_plan_t **out) {
    return plan_create(n, m, dtype, nullptr, out);
}

int pa_final_key_length(uint64_t n, uint64_t t, uint64_t s, uint64_t *r) {
    if (!r) return PA_EINVAL;
    *r = 0;
    if (t >= n || s >= n - t) return PA_EINVAL;  // Eq. 1 needs r = n - t - s >= 1
    *r = n - t - s;
    return PA_OK;
}

double pa_leakage_bound(uint64_t n, uint64_t t, uint64_t r) {
    // Eq. 1: I(K; g, V) <= 2^-s / ln 2 with s = n - t - r (may be <= 0: then the bound is >= 1/ln 2)
    const double s = (double)n - (double)t - (double)r;
    return std::exp2(-s) / std::log(2.0);
}

int pa_plan_modified(uint64_t n, uint64_t m, pa_dtype_t dtype, pa_plan_t **out) {
    return plan_create(n, m, dtype, nullptr, out, true);
}

int pa_plan_splits(uint64_t n, uint64_t m, pa_dtype_t dtype, uint32_t *L1, uint32_t *L2, uint32_t *L3, int cap,
                   int *count) {
    if (!count || cap < 0 || (cap > 0 && (!L1 || !L2 || !L3))) return PA_EINVAL;
    *count = 0;
    if (!plan_args_ok(n, m, dtype)) return PA_EINVAL;
    const Geometry geo = choose_geometry(n + m - 1, dtype, false);
    if (geo.L == 0) return PA_EUNSUPPORTED;
    const std::vector<Geometry> cand = geometry_candidates(geo.L, dtype, false);
    int c = 0;
    for (const Geometry &g : cand) {
        if (c < cap) split_lengths(g, &L1[c], &L2[c], &L3[c]);
        ++c;
    }
    *count = c;
    return PA_OK;
}

int pa_plan_split(uint64_t n, uint64_t m, pa_dtype_t dtype, uint32_t L1, uint32_t L2, uint32_t L3, pa_plan_t **out) {
    if (!out) return PA_EINVAL;
    *out = nullptr;
    if (!plan_args_ok(n, m, dtype)) return PA_EINVAL;
    const Geometry geo = choose_geometry(n + m - 1, dtype, false);
    if (geo.L == 0) return PA_EUNSUPPORTED;
    for (const Geometry &g : geometry_candidates(geo.L, dtype, false)) {
        uint32_t a, b, c;
        split_lengths(g, &a, &b, &c);
        if (a == L1 && b == L2 && c == L3) return plan_create(n, m, dtype, &g, out);
    }
    return PA_EINVAL;
}

int pa_plan_destroy(pa_plan_t *plan) {
    if (!plan) return PA_OK;
    DeviceGuard g(plan->device);
    cudaDeviceSynchronize();
    free_plan(plan);
    return PA_OK;
}

int pa_plan_shape(const pa_plan_t *p, uint64_t *L, uint32_t *L1, uint32_t *L2, uint32_t *L3) {
    if (!p) return PA_EINVAL;
    if (L) *L = p->L;
    uint32_t a, b, c;
    split_lengths(p->geo, &a, &b, &c);
    if (L1) *L1 = a;
    if (L2) *L2 = b;
    if (L3) *L3 = c;
    return PA_OK;
}

int pa_plan_set_guard(pa_plan_t *p, float threshold) {
    if (!p) return PA_EINVAL;
    p->guard = threshold;
    return PA_OK;
}

int pa_plan_set_staged(pa_plan_t *p, int on) {
    if (!p) return PA_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    p->staged = on != 0;
    return PA_OK;
}

int pa_plan_set_storage_bits(pa_plan_t *p, uint32_t bits) {
    if (!p || bits > 23) return PA_EINVAL;
    if (p->dtype != PA_FP32_GUARD) return PA_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(p->mu);
    p->store_bits = (bits == 23) ? 0u : bits;
    p->seeded = false;  // the cached spectrum was stored at the old width: pa_set_seed again
    return PA_OK;
}

int pa_plan_expire_waits(pa_plan_t *p, uint32_t launches) {
    if (!p) return PA_EINVAL;
    const Geometry &g = p->geo;
    if (!p->staged || p->dtype != PA_FP32_GUARD || !inv_bits_staged(elem_bytes(p->dtype), g.lg1))
        return PA_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(p->mu);
    p->expire_launches = launches;
    return PA_OK;
}

int pa_profile_enable(pa_plan_t *p, int enable) {
    if (!p) return PA_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    p->prof = enable != 0;
    return PA_OK;
}

int pa_profile_read(pa_plan_t *p, pa_kernel_stat_t *stats, int *count, int reset) {
    if (!p || !stats || !count) return PA_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard g(p->device);
    collect_events(p);
    int c = 0;
    for (int k = 0; k < PA_NUM_KERNEL_KINDS; ++k) {
        stats[c].name = kKindNames[k];
        stats[c].launches = p->launches[k];
        stats[c].total_ms = p->total_ms[k];
        ++c;
        if (reset) {
            p->launches[k] = 0;
            p->total_ms[k] = 0.0;
        }
    }
    *count = c;
    return PA_OK;
}

int pa_set_seed(pa_plan_t *p, const uint64_t *seed_dev, uint64_t seed_bits, pa_stream_t stream) {
    if (!p || !seed_dev || !aligned16(seed_dev)) return PA_EINVAL;
    if (seed_bits != p->n + p->m - 1) return PA_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard g(p->device);
    if (!g.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = ensure_work(p, 1);
    if (rc != PA_OK) return rc;
    if (!p->done) PA_CUDA(cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming));
    PA_CUDA(cudaStreamWaitEvent(st, p->done, 0));  // after the plan's previous work, on any stream
    const size_t sw = (size_t)((seed_bits + 63) / 64);
    if (!p->seed_copy) PA_CUDA(cudaMalloc(&p->seed_copy, sw * sizeof(uint64_t)));
    PA_CUDA(cudaMemcpyAsync(p->seed_copy, seed_dev, sw * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    rc = (p->dtype == PA_FP32_GUARD) ? run_seed<float>(p, p->seed_copy, st)
         : (p->dtype == PA_FP64)     ? run_seed<double>(p, p->seed_copy, st)
                                     : run_seed<Zp>(p, p->seed_copy, st);
    if (rc != PA_OK) return rc;
    if (p->real) {
        p->real->seeded = false;
        rc = (p->dtype == PA_FP32_GUARD) ? run_seed_real<float>(p, p->seed_copy, st)
                                         : run_seed_real<double>(p, p->seed_copy, st);
        if (rc != PA_OK) return rc;
        p->real->seeded = true;
    }
    PA_CUDA(cudaEventRecord(p->done, st));
    p->seeded = true;
    if (p->fallback) p->fallback->seeded = false;  // re-seeded lazily on the next escalation
    return PA_OK;
}

int pa_hash_batch_async(pa_plan_t *p, const uint64_t *keys_dev, uint32_t nkeys, uint64_t key_stride_words,
                        uint64_t *out_dev, uint64_t out_stride_words, pa_stream_t stream) {
    if (!p || !keys_dev || !out_dev || nkeys == 0) return PA_EINVAL;
    if (!aligned16(keys_dev) || !aligned16(out_dev)) return PA_EINVAL;
    if (key_stride_words < (p->n_key + 63) / 64 || out_stride_words < (p->m + 63) / 64) return PA_EINVAL;
    if ((nkeys > 1 && (key_stride_words & 1)) || (nkeys > 1 && (out_stride_words & 1))) return PA_EINVAL;
    if (!p->seeded) return PA_ENOSEED;
    std::lock_guard<std::mutex> lk(p->mu);
    if (p->pending.active) return PA_EAGAIN;
    DeviceGuard g(p->device);
    if (!g.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = issue_batch(p, keys_dev, nkeys, key_stride_words, out_dev, out_stride_words, st);
    if (rc != PA_OK) return rc;
    PA_CUDA(cudaEventRecord(p->done, st));
    PendingBatch b;
    b.active = true;
    b.keys = keys_dev;
    b.nkeys = nkeys;
    b.kstride = key_stride_words;
    b.out = out_dev;
    b.ostride = out_stride_words;
    b.stream = stream;
    p->pending = b;
    return PA_OK;
}

int pa_hash_host_async(pa_plan_t *p, const uint64_t *keys_host, uint32_t nkeys, uint64_t key_stride_words,
                       uint64_t *out_host, uint64_t out_stride_words, pa_stream_t stream) {
    if (!p || !keys_host || !out_host || nkeys == 0) return PA_EINVAL;
    const uint64_t kw = (p->n_key + 63) / 64, ow = (p->m + 63) / 64;
    if (key_stride_words < kw || out_stride_words < ow) return PA_EINVAL;
    if (!p->seeded) return PA_ENOSEED;
    std::lock_guard<std::mutex> lk(p->mu);
    if (p->pending.active) return PA_EAGAIN;
    DeviceGuard g(p->device);
    if (!g.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t dks = kw + (kw & 1), dos = ow + (ow & 1);  // even device strides: 16-byte aligned rows
    int rc = ensure_staging(p, (size_t)nkeys * dks, (size_t)nkeys * dos);
    if (rc != PA_OK) return rc;
    // keys in on their own stream, so they can overlap the compute of the batch before
    PA_CUDA(cudaMemcpy2DAsync(p->stage_keys, dks * sizeof(uint64_t), keys_host, key_stride_words * sizeof(uint64_t),
                              kw * sizeof(uint64_t), nkeys, cudaMemcpyHostToDevice, p->s_in));
    PA_CUDA(cudaEventRecord(p->ev_in, p->s_in));
    PA_CUDA(cudaStreamWaitEvent(st, p->ev_in, 0));
    rc = issue_batch(p, p->stage_keys, nkeys, dks, p->stage_out, dos, st);
    if (rc != PA_OK) return rc;
    // final keys out on a third stream, so they overlap the compute of the batch after
    PA_CUDA(cudaEventRecord(p->ev_comp, st));
    PA_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_comp, 0));
    PA_CUDA(cudaMemcpy2DAsync(out_host, out_stride_words * sizeof(uint64_t), p->stage_out, dos * sizeof(uint64_t),
                              ow * sizeof(uint64_t), nkeys, cudaMemcpyDeviceToHost, p->s_out));
    PA_CUDA(cudaEventRecord(p->done, p->s_out));
    PendingBatch b;
    b.active = true;
    b.keys = p->stage_keys;
    b.nkeys = nkeys;
    b.kstride = dks;
    b.out = p->stage_out;
    b.ostride = dos;
    b.stream = stream;
    b.host_out = out_host;
    b.host_ostride = out_stride_words;
    p->pending = b;
    return PA_OK;
}

int pa_hash_host(pa_plan_t *p, const uint64_t *keys_host, uint32_t nkeys, uint64_t key_stride_words, uint64_t *out_host,
                 uint64_t out_stride_words, pa_stream_t stream, pa_batch_info_t *info) {
    int rc = pa_hash_host_async(p, keys_host, nkeys, key_stride_words, out_host, out_stride_words, stream);
    if (rc != PA_OK) return rc;
    return pa_batch_finish(p, info);
}

int pa_batch_finish(pa_plan_t *p, pa_batch_info_t *info) {
    if (!p) return PA_EINVAL;
    std::unique_lock<std::mutex> lk(p->mu);
    if (!p->pending.active) return PA_EINVAL;
    const PendingBatch b = p->pending;
    p->pending.active = false;
    DeviceGuard g(p->device);
    if (!g.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    PA_CUDA(cudaEventSynchronize(p->done));
    uint32_t err_word = 0;
    std::memcpy(&err_word, p->h_marg + b.nkeys, sizeof(uint32_t));
    if (err_word != 0) {
        PA_CUDA(cudaMemset(p->err, 0, sizeof(uint32_t)));
        // this batch's outputs are not valid: bit 0, a bounded device wait ran out; bit 1, a
        // staging buffer was not aligned for its tiled copy (the kernel copied nothing)
        if (err_word & 1u) return PA_ETIMEOUT;
        g_last_cuda_error = "device staging buffer misaligned for its tiled copy";
        return PA_ECUDA;
    }
    if (info) info->escalated = 0;
    uint32_t escalated = 0;
    for (uint32_t k = 0; k < b.nkeys; ++k) {
        float mk_ = p->h_marg[k];
        int32_t mode = (int32_t)p->dtype;
        if (p->dtype == PA_FP32_GUARD && !(mk_ <= p->guard)) {
            // Recompute this key one mode wider (the guard's escalation): FP32 -> FP64 (-> exact NTT
            // inside the FP64 plan when its own margin fails).
            if (!p->fallback) {
                pa_plan_t *fb = nullptr;
                int rc = plan_create(p->n_key, p->m, PA_FP64, nullptr, &fb, p->modified);
                if (rc != PA_OK) return rc;
                p->fallback = fb;
            }
            int rc = escalate_key(p, b, k, &mk_, &mode);
            if (rc != PA_OK) return rc;
            ++escalated;
        } else if (p->dtype == PA_FP64 && !(mk_ <= p->guard)) {
            if (!p->fallback) {
                pa_plan_t *fb = nullptr;
                int rc = plan_create(p->n_key, p->m, PA_NTT64, nullptr, &fb, p->modified);
                if (rc != PA_OK) return rc;
                p->fallback = fb;
            }
            int rc = escalate_key(p, b, k, &mk_, &mode);
            if (rc != PA_OK) return rc;
            ++escalated;
        }
        if (info && info->margin) info->margin[k] = mk_;
        if (info && info->mode) info->mode[k] = mode;
    }
    if (info) info->escalated = escalated;
    return PA_OK;
}

int pa_hash_batch(pa_plan_t *p, const uint64_t *keys_dev, uint32_t nkeys, uint64_t key_stride_words,
                  uint64_t *out_dev, uint64_t out_stride_words, pa_stream_t stream, pa_batch_info_t *info) {
    int rc = pa_hash_batch_async(p, keys_dev, nkeys, key_stride_words, out_dev, out_stride_words, stream);
    if (rc != PA_OK) return rc;
    const bool need_margins = (p->dtype == PA_FP32_GUARD) || info != nullptr;
    if (!need_margins) {
        // FP64 and NTT64 without diagnostics return right after issuing: the batch completes in
        // stream order, and the error word is examined by the next call that waits.
        std::lock_guard<std::mutex> lk(p->mu);
        p->pending.active = false;
        return PA_OK;
    }
    return pa_batch_finish(p, info);
}

}  // extern "C"

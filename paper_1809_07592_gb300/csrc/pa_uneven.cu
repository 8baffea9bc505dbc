// pa_uneven.cu -- uneven batches: blocks of different (n, m), each with its own seed.
//
// Blocks are grouped into classes by transform length L, the smallest smooth
// length ro * 2^k >= n+m-1 (ro in {1, 3, 5, 9}; powers of two in the exact mode).
// Complex modes use the paper's real-valued FFT acceleration (Eq. 5-10): key and
// seed of a block ride in one complex transform z = x + i*sigma, the fused
// innermost pass separates their spectra from the bin pair (k, -k), multiplies
// them, and sends two blocks' products through one inverse as Y1 + i*Y2. The
// whole schedule can be captured once into a CUDA graph whose branches (one per
// class) run concurrently; replaying it costs one graph launch.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "pa.h"
#include "pa_blocks.h"
#include "pa_internal.h"
#include "pa_kernels.cuh"
#include "pa_launch.h"

using namespace pa;
using pa::blocks::ClassRun;

namespace {

#define U_CUDA(call)                                                     \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return pa_internal_cuda_fail(e_, #call);  \
    } while (0)

struct UClass {
    Geometry geo;                    // length L and the chosen split
    std::vector<uint32_t> ids;       // caller indices of the blocks in this class
    BlockDev *d_blocks = nullptr;    // device descriptors
    void *Wf = nullptr, *Wi = nullptr;  // forward slots (one per block), inverse slots (one per pair)
    void *spec = nullptr;            // NTT mode: one seed-spectrum slot, blocks run one after another
    void *tw_hi = nullptr, *tw_lo = nullptr;
    uint32_t B = 0;
    void *tw_fine = nullptr;         // stage twiddles, length geo.F() (rebuilt when the split changes F)
    uint32_t fineF = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    ClassRun run(const Geometry &g) const {
        ClassRun r;
        r.geo = g;
        r.d_blocks = d_blocks;
        r.nb = (uint32_t)ids.size();
        r.Wf = Wf;
        r.Wi = Wi;
        r.spec = spec;
        r.tw_hi = tw_hi;
        r.tw_lo = tw_lo;
        r.B = B;
        r.tw_fine = tw_fine;
        return r;
    }
};

// ---------------------------------------------------------------------------
// Autotuner cache: best split per (L, dtype), measured on the first batch that needs it.
std::mutex g_tune_mu;
std::map<std::pair<uint64_t, int>, Geometry> g_tune;
bool g_tune_loaded = false;

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("PA_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    unsigned long long L;
    int dt, a, b, ro, lgI;
    while (std::fscanf(f, "%llu %d %d %d %d %d", &L, &dt, &a, &b, &ro, &lgI) == 6)
        g_tune[{(uint64_t)L, dt}] = Geometry{(uint64_t)L, a, b, ro, lgI};
    std::fclose(f);
}

}  // namespace

struct pa_uneven {
    pa_dtype_t dtype = PA_FP32_GUARD;
    int device = 0;
    uint32_t nblocks = 0;
    std::vector<pa_block_desc_t> blocks;
    std::vector<UClass> classes;
    uint32_t *popc = nullptr, *marg = nullptr;
    float *h_marg = nullptr;
    float guard = 0.25f;
    bool use_graph = false;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::map<std::pair<uint64_t, uint64_t>, pa_plan_t *> esc;  // escalation plans by (n, m)
    std::mutex mu;
};

namespace {

template <typename T>
TwTab<T> tw_of(const ClassRun &c) {
    TwTab<T> t;
    t.hi = static_cast<const cx<T> *>(c.tw_hi);
    t.lo = static_cast<const cx<T> *>(c.tw_lo);
    t.B = c.B;
    t.lgL = 0;
    while ((1ull << t.lgL) < c.geo.L) ++t.lgL;
    t.fine = static_cast<const cx<T> *>(c.tw_fine);
    t.F = c.geo.F();
    return t;
}

// Middle strided pass over `slots` consecutive slots, chunked to the grid's y limit.
template <typename T>
int mid_chunks(const ClassRun &c, bool inverse, cx<T> *W, uint32_t slots, cudaStream_t st) {
    const uint32_t nblk = 1u << c.geo.lg1;
    const uint32_t per = 65535u / nblk;
    const TwTab<T> tw = tw_of<T>(c);
    for (uint32_t s0 = 0; s0 < slots; s0 += per) {
        const uint32_t k = (slots - s0 < per) ? slots - s0 : per;
        U_CUDA(launch_mid<T>(c.geo.lgM, inverse, W + (uint64_t)s0 * c.geo.L, c.geo.L, c.geo.inner(), k, tw, st));
    }
    return PA_OK;
}

// The whole chain of one class (complex modes).
template <typename T>
int run_class_complex(const ClassRun &c, uint32_t *popc, uint32_t *marg, cudaStream_t st) {
    const Geometry &g = c.geo;
    const uint32_t nb = c.nb;
    const TwTab<T> tw = tw_of<T>(c);
    cx<T> *Wf = static_cast<cx<T> *>(c.Wf), *Wi = static_cast<cx<T> *>(c.Wi);
    U_CUDA(launch_zero_blocks(c.d_blocks, nb, popc, marg, st));
    U_CUDA(launch_fwd_keyseed<T>(g.lg1, c.d_blocks, nb, Wf, g.L, tw, popc, st));
    if (g.lgM) {
        int rc = mid_chunks<T>(c, false, Wf, nb, st);
        if (rc != PA_OK) return rc;
    }
    U_CUDA(launch_middle_split<T>(g.ro, g.lgI, Wf, Wi, g.L, nb, (uint32_t)g.lg1, (uint32_t)g.lgM, tw, st));
    if (g.lgM) {
        int rc = mid_chunks<T>(c, true, Wi, (nb + 1) / 2, st);
        if (rc != PA_OK) return rc;
    }
    U_CUDA(launch_inv_bits_blocks<T>(g.lg1, Wi, g.L, c.d_blocks, nb, popc, marg, tw, st));
    return PA_OK;
}

// NTT mode: per block, seed transform into the class's spectrum slot, then the key.
int run_class_ntt(const ClassRun &c, const pa_block_desc_t *hb, const uint32_t *ids, uint32_t *popc,
                  uint32_t *marg, cudaStream_t st) {
    const TwTab<Zp> tw = tw_of<Zp>(c);
    cx<Zp> *W = static_cast<cx<Zp> *>(c.Wf), *spec = static_cast<cx<Zp> *>(c.spec);
    const Geometry &g = c.geo;
    const uint64_t L = g.L;
    const cx<Zp> invL = zp_pow2(192 - (int)tw.lgL);  // L^-1 mod p = 2^(192 - log2 L)
    for (uint32_t i = 0; i < c.nb; ++i) {
        const pa_block_desc_t &b = hb[ids[i]];
        const uint64_t kw = (b.n + 63) / 64;
        U_CUDA(launch_fwd_seed<Zp>(g.lg1, b.seed, b.n, b.m, W, L, tw, st));
        if (g.lgM) U_CUDA(launch_mid<Zp>(g.lgM, false, W, L, g.inner(), 1, tw, st));
        U_CUDA(launch_middle<Zp>(g.ro, g.lgI, 1, W, spec, L, 1, tw, invL, st));
        U_CUDA(launch_zero_keys(1, popc + ids[i], marg + ids[i], st));
        U_CUDA(launch_fwd_keys<Zp>(g.lg1, b.key, 1, kw, b.n, W, L, 1, tw, popc + ids[i], st));
        if (g.lgM) U_CUDA(launch_mid<Zp>(g.lgM, false, W, L, g.inner(), 1, tw, st));
        U_CUDA(launch_middle<Zp>(g.ro, g.lgI, 0, W, spec, L, 1, tw, (cx<Zp>)1, st));
        if (g.lgM) U_CUDA(launch_mid<Zp>(g.lgM, true, W, L, g.inner(), 1, tw, st));
        U_CUDA(launch_inv_bits<Zp>(g.lg1, W, L, b.m, 1, popc + ids[i], marg + ids[i], b.out, (b.m + 63) / 64, 1, tw,
                                   st));
    }
    return PA_OK;
}

int run_class(pa_uneven_t *u, const UClass &c, cudaStream_t st) {
    if (u->dtype == PA_NTT64) return run_class_ntt(c.run(c.geo), u->blocks.data(), c.ids.data(), u->popc, u->marg, st);
    return pa::blocks::run_complex(u->dtype, c.run(c.geo), u->popc, u->marg, st);
}

// (Re)build the stage-twiddle table of a class for the F of its current split.
int class_fine(pa_uneven_t *u, UClass &c) {
    const uint32_t F = c.geo.F();
    if (c.tw_fine && c.fineF == F) return PA_OK;
    if (c.tw_fine) cudaFree(c.tw_fine);
    c.tw_fine = nullptr;
    void *hi = nullptr, *lo = nullptr;
    uint32_t B = 0;
    int rc = pa_internal_twiddles(c.geo.L, F, (int)u->dtype, &hi, &lo, &B, &c.tw_fine);
    if (rc != PA_OK) return rc;
    cudaFree(hi);
    cudaFree(lo);
    c.fineF = F;
    return PA_OK;
}

// Choose a class's split: cached, else time every candidate on the class's own data.
int tune_class(pa_uneven_t *u, UClass &c) {
    const uint64_t L = c.geo.L;
    std::vector<Geometry> cand = pa::blocks::candidates(L, u->dtype);
    if (cand.empty()) return PA_EUNSUPPORTED;
    if (pa::blocks::cached_split(L, u->dtype, &c.geo)) return class_fine(u, c);
    if (cand.size() == 1 || u->dtype == PA_NTT64) {
        c.geo = pa::blocks::default_split(L, u->dtype);
        pa::blocks::store_split(c.geo, u->dtype);
        return class_fine(u, c);
    }
    cudaEvent_t a, b;
    U_CUDA(cudaEventCreate(&a));
    U_CUDA(cudaEventCreate(&b));
    float best = 1e30f;
    Geometry bestg = cand[0];
    for (const Geometry &g : cand) {
        c.geo = g;
        int rc = class_fine(u, c);
        if (rc != PA_OK) return rc;
        float total = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            U_CUDA(cudaEventRecord(a, c.st));
            rc = pa::blocks::run_complex(u->dtype, c.run(g), u->popc, u->marg, c.st);
            if (rc != PA_OK) return rc;
            U_CUDA(cudaEventRecord(b, c.st));
            U_CUDA(cudaEventSynchronize(b));
            float ms = 0.f;
            U_CUDA(cudaEventElapsedTime(&ms, a, b));
            if (rep > 0) total += ms;  // the first run warms up
        }
        if (total < best) {
            best = total;
            bestg = g;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c.geo = bestg;
    pa::blocks::store_split(c.geo, u->dtype);
    return class_fine(u, c);
}

void free_uneven(pa_uneven_t *u) {
    if (!u) return;
    if (u->exec) cudaGraphExecDestroy(u->exec);
    if (u->graph) cudaGraphDestroy(u->graph);
    for (UClass &c : u->classes) {
        cudaFree(c.d_blocks);
        cudaFree(c.Wf);
        cudaFree(c.Wi);
        cudaFree(c.spec);
        cudaFree(c.tw_hi);
        cudaFree(c.tw_lo);
        cudaFree(c.tw_fine);
        if (c.st) cudaStreamDestroy(c.st);
        if (c.done) cudaEventDestroy(c.done);
    }
    for (auto &kv : u->esc) pa_plan_destroy(kv.second);
    cudaFree(u->popc);
    cudaFree(u->marg);
    if (u->h_marg) cudaFreeHost(u->h_marg);
    if (u->fork) cudaEventDestroy(u->fork);
    if (u->cap) cudaStreamDestroy(u->cap);
    delete u;
}

uint64_t block_length(const pa_block_desc_t &b, pa_dtype_t dtype) {
    return pa::blocks::class_length(b.n, b.m, dtype);
}

bool desc_ok(const pa_block_desc_t &b) {
    if (b.n == 0 || b.m == 0 || b.m > b.n || b.n > (1ull << 27)) return false;
    if (!b.key || !b.seed || !b.out) return false;
    return ((reinterpret_cast<uintptr_t>(b.key) | reinterpret_cast<uintptr_t>(b.seed) |
             reinterpret_cast<uintptr_t>(b.out)) & 15u) == 0;
}

std::vector<BlockDev> class_descs(const pa_uneven_t *u, const UClass &c) {
    std::vector<BlockDev> v(c.ids.size());
    for (size_t i = 0; i < c.ids.size(); ++i) {
        const pa_block_desc_t &b = u->blocks[c.ids[i]];
        v[i] = BlockDev{b.n, b.m, b.key, b.seed, b.out, c.ids[i], 0u};
    }
    return v;
}

int record_all(pa_uneven_t *u, cudaStream_t st) {
    for (const UClass &c : u->classes) {
        int rc = run_class(u, c, st);
        if (rc != PA_OK) return rc;
    }
    return PA_OK;
}

int capture_graph(pa_uneven_t *u) {
    U_CUDA(cudaStreamBeginCapture(u->cap, cudaStreamCaptureModeThreadLocal));
    int rc = PA_OK;
    cudaError_t e = cudaEventRecord(u->fork, u->cap);
    for (UClass &c : u->classes) {
        if (e != cudaSuccess || rc != PA_OK) break;
        e = cudaStreamWaitEvent(c.st, u->fork, 0);
        if (e == cudaSuccess) rc = run_class(u, c, c.st);
        if (e == cudaSuccess && rc == PA_OK) e = cudaEventRecord(c.done, c.st);
        if (e == cudaSuccess && rc == PA_OK) e = cudaStreamWaitEvent(u->cap, c.done, 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(u->cap, &g);
    if (e != cudaSuccess) return pa_internal_cuda_fail(e, "capture");
    if (rc != PA_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e2 != cudaSuccess) return pa_internal_cuda_fail(e2, "cudaStreamEndCapture");
    u->graph = g;
    U_CUDA(cudaGraphInstantiate(&u->exec, g, 0));
    return PA_OK;
}

}  // namespace

namespace pa {
namespace blocks {

uint64_t class_length(uint64_t n, uint64_t m, pa_dtype_t dtype) {
    return choose_geometry(n + m - 1, dtype, dtype != PA_NTT64).L;
}

size_t scratch_per_block(uint64_t L, pa_dtype_t dtype) {
    if (dtype == PA_NTT64) return 2 * L * 8;
    const size_t e = dtype == PA_FP32_GUARD ? sizeof(float2) : sizeof(double2);
    return L * e + (L * e + 1) / 2 + sizeof(BlockDev) + 8;  // forward slot, half an inverse slot, descriptor, counters
}

int run_complex(pa_dtype_t dtype, const ClassRun &c, uint32_t *popc, uint32_t *marg, cudaStream_t st) {
    return dtype == PA_FP32_GUARD ? run_class_complex<float>(c, popc, marg, st)
                                  : run_class_complex<double>(c, popc, marg, st);
}

int run_ntt(const ClassRun &c, const pa_block_desc_t *hb, const uint32_t *ids, uint32_t *popc, uint32_t *marg,
            cudaStream_t st) {
    return run_class_ntt(c, hb, ids, popc, marg, st);
}

std::vector<Geometry> candidates(uint64_t L, pa_dtype_t dtype) {
    return geometry_candidates(L, dtype, dtype != PA_NTT64);
}

Geometry default_split(uint64_t L, pa_dtype_t dtype) { return default_geometry(L, dtype, dtype != PA_NTT64); }

bool cached_split(uint64_t L, pa_dtype_t dtype, Geometry *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find({L, (int)dtype});
    if (it == g_tune.end()) return false;
    *out = it->second;
    return true;
}

void store_split(const Geometry &g, pa_dtype_t dtype) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[{g.L, (int)dtype}] = g;
    const char *path = std::getenv("PA_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%llu %d %d %d %d %d\n", (unsigned long long)g.L, (int)dtype, g.lg1, g.lgM, g.ro, g.lgI);
    std::fclose(f);
}

}  // namespace blocks
}  // namespace pa

extern "C" {

int pa_uneven_create(const pa_block_desc_t *blocks, uint32_t nblocks, pa_dtype_t dtype, int use_graph,
                     pa_uneven_t **out) {
    if (!out || !blocks || nblocks == 0) return PA_EINVAL;
    *out = nullptr;
    if (dtype != PA_FP32_GUARD && dtype != PA_FP64 && dtype != PA_NTT64) return PA_EINVAL;
    for (uint32_t i = 0; i < nblocks; ++i)
        if (!desc_ok(blocks[i])) return PA_EINVAL;
    for (uint32_t i = 0; i < nblocks; ++i)
        if (block_length(blocks[i], dtype) == 0) return PA_EUNSUPPORTED;
    pa_uneven_t *u = new pa_uneven_t();
    u->dtype = dtype;
    u->nblocks = nblocks;
    u->use_graph = use_graph != 0;
    u->blocks.assign(blocks, blocks + nblocks);
    cudaGetDevice(&u->device);
    std::map<uint64_t, std::vector<uint32_t>> byL;
    for (uint32_t i = 0; i < nblocks; ++i) byL[block_length(blocks[i], dtype)].push_back(i);
    const size_t esz = dtype == PA_FP32_GUARD ? sizeof(float2) : dtype == PA_FP64 ? sizeof(double2) : 8;
    int rc = PA_OK;
    auto fail = [&](int r) {
        free_uneven(u);
        return r;
    };
#define U_TRY(call)                                                                       \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ == cudaErrorMemoryAllocation) { cudaGetLastError(); return fail(PA_ENOMEM); } \
        if (e_ != cudaSuccess) return fail(pa_internal_cuda_fail(e_, #call));             \
    } while (0)
    U_TRY(cudaMalloc(&u->popc, nblocks * sizeof(uint32_t)));
    U_TRY(cudaMalloc(&u->marg, nblocks * sizeof(uint32_t)));
    U_TRY(cudaMallocHost(&u->h_marg, nblocks * sizeof(float)));
    U_TRY(cudaStreamCreateWithFlags(&u->cap, cudaStreamNonBlocking));
    U_TRY(cudaEventCreateWithFlags(&u->fork, cudaEventDisableTiming));
    for (auto &kv : byL) {
        UClass c;
        c.geo = pa::blocks::default_split(kv.first, dtype);
        c.ids = kv.second;
        u->classes.push_back(c);
    }
    for (UClass &c : u->classes) {
        const uint32_t nb = (uint32_t)c.ids.size();
        U_TRY(cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking));
        U_TRY(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
        std::vector<BlockDev> d = class_descs(u, c);
        U_TRY(cudaMalloc(&c.d_blocks, d.size() * sizeof(BlockDev)));
        U_TRY(cudaMemcpy(c.d_blocks, d.data(), d.size() * sizeof(BlockDev), cudaMemcpyHostToDevice));
        const uint64_t L = c.geo.L;
        if (dtype == PA_NTT64) {
            U_TRY(cudaMalloc(&c.Wf, L * esz));
            U_TRY(cudaMalloc(&c.spec, L * esz));
        } else {
            U_TRY(cudaMalloc(&c.Wf, (size_t)nb * L * esz));
            U_TRY(cudaMalloc(&c.Wi, (size_t)((nb + 1) / 2) * L * esz));
        }
        rc = pa_internal_twiddles(L, c.geo.F(), (int)dtype, &c.tw_hi, &c.tw_lo, &c.B, &c.tw_fine);
        if (rc != PA_OK) return fail(rc);
        c.fineF = c.geo.F();
        rc = tune_class(u, c);
        if (rc != PA_OK) return fail(rc);
    }
    U_TRY(cudaDeviceSynchronize());
    if (u->use_graph) {
        // one direct run first, so every kernel instance is loaded and configured before capture
        rc = record_all(u, u->cap);
        if (rc != PA_OK) return fail(rc);
        U_TRY(cudaStreamSynchronize(u->cap));
        rc = capture_graph(u);
        if (rc != PA_OK) return fail(rc);
    }
#undef U_TRY
    *out = u;
    return PA_OK;
}

int pa_uneven_update(pa_uneven_t *u, const pa_block_desc_t *blocks, uint32_t nblocks, pa_stream_t stream) {
    if (!u || !blocks || nblocks != u->nblocks) return PA_EINVAL;
    for (uint32_t i = 0; i < nblocks; ++i) {
        if (!desc_ok(blocks[i]) || blocks[i].n != u->blocks[i].n || blocks[i].m != u->blocks[i].m) return PA_EINVAL;
    }
    std::lock_guard<std::mutex> lk(u->mu);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    u->blocks.assign(blocks, blocks + nblocks);
    if (u->dtype == PA_NTT64 && u->use_graph) {
        // the NTT chains bake block pointers into the launches: capture again
        if (u->exec) cudaGraphExecDestroy(u->exec);
        if (u->graph) cudaGraphDestroy(u->graph);
        u->exec = nullptr;
        u->graph = nullptr;
        U_CUDA(cudaStreamSynchronize(st));
        return capture_graph(u);
    }
    for (UClass &c : u->classes) {
        std::vector<BlockDev> d = class_descs(u, c);
        U_CUDA(cudaMemcpyAsync(c.d_blocks, d.data(), d.size() * sizeof(BlockDev), cudaMemcpyHostToDevice, st));
    }
    U_CUDA(cudaStreamSynchronize(st));  // the host copies above live on this stack frame
    return PA_OK;
}

int pa_uneven_run(pa_uneven_t *u, pa_stream_t stream, pa_batch_info_t *info) {
    if (!u) return PA_EINVAL;
    std::lock_guard<std::mutex> lk(u->mu);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (u->exec) {
        U_CUDA(cudaGraphLaunch(u->exec, st));
    } else {
        int rc = record_all(u, st);
        if (rc != PA_OK) return rc;
    }
    if (info) info->escalated = 0;
    if (u->dtype != PA_FP32_GUARD && !info) return PA_OK;
    U_CUDA(cudaMemcpyAsync(u->h_marg, u->marg, u->nblocks * sizeof(float), cudaMemcpyDeviceToHost, st));
    U_CUDA(cudaStreamSynchronize(st));
    uint32_t escalated = 0;
    for (uint32_t i = 0; i < u->nblocks; ++i) {
        float mg = u->h_marg[i];
        int32_t mode = (int32_t)u->dtype;
        if (u->dtype != PA_NTT64 && !(mg <= u->guard)) {
            // recompute this block one mode wider through a per-(n, m) plan
            const pa_block_desc_t &b = u->blocks[i];
            const pa_dtype_t wider = u->dtype == PA_FP32_GUARD ? PA_FP64 : PA_NTT64;
            auto key = std::make_pair(b.n, b.m);
            auto it = u->esc.find(key);
            pa_plan_t *pl = nullptr;
            if (it == u->esc.end()) {
                int rc = pa_plan(b.n, b.m, wider, &pl);
                if (rc != PA_OK) return rc;
                u->esc[key] = pl;
            } else {
                pl = it->second;
            }
            int rc = pa_set_seed(pl, b.seed, b.n + b.m - 1, stream);
            if (rc != PA_OK) return rc;
            float m2 = 0.f;
            int32_t mode2 = 0;
            pa_batch_info_t sub{&m2, &mode2, 0, 0};
            rc = pa_hash_batch(pl, b.key, 1, (b.n + 63) / 64, b.out, (b.m + 63) / 64, stream, &sub);
            if (rc != PA_OK) return rc;
            mg = m2;
            mode = mode2;
            ++escalated;
        }
        if (info && info->margin) info->margin[i] = mg;
        if (info && info->mode) info->mode[i] = mode;
    }
    if (info) info->escalated = escalated;
    return PA_OK;
}

int pa_uneven_set_guard(pa_uneven_t *u, float threshold) {
    if (!u) return PA_EINVAL;
    u->guard = threshold;
    return PA_OK;
}

int pa_uneven_destroy(pa_uneven_t *u) {
    if (!u) return PA_OK;
    cudaDeviceSynchronize();
    free_uneven(u);
    return PA_OK;
}

int pa_uneven_class(const pa_uneven_t *u, uint32_t c, uint32_t *nclasses, uint64_t *L, uint32_t *L1, uint32_t *L2,
                    uint32_t *L3, uint32_t *nb) {
    if (!u) return PA_EINVAL;
    if (nclasses) *nclasses = (uint32_t)u->classes.size();
    if (c >= u->classes.size()) return (nclasses && !L && !L1 && !L2 && !L3 && !nb) ? PA_OK : PA_EINVAL;
    const UClass &k = u->classes[c];
    if (L) *L = k.geo.L;
    if (L1) *L1 = 1u << k.geo.lg1;
    if (L2) *L2 = k.geo.lgM ? (1u << k.geo.lgM) : k.geo.inner();
    if (L3) *L3 = k.geo.lgM ? k.geo.inner() : 1u;
    if (nb) *nb = (uint32_t)k.ids.size();
    return PA_OK;
}

int pa_hash_uneven(const pa_block_desc_t *blocks, uint32_t nblocks, pa_dtype_t dtype, pa_stream_t stream,
                   pa_batch_info_t *info) {
    pa_uneven_t *u = nullptr;
    int rc = pa_uneven_create(blocks, nblocks, dtype, 0, &u);
    if (rc != PA_OK) return rc;
    rc = pa_uneven_run(u, stream, info);
    cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    pa_uneven_destroy(u);
    return rc;
}

}  // extern "C"

// pa_server.cu -- the serving loop: continuous batching of privacy-amplification
// blocks as reconciliation emits them.
//
// pa_submit queues a block and returns a ticket. One worker thread per server
// admits queued blocks in arrival order while the device scratch of everything
// in flight stays under the HBM admission cap, groups each admitted micro-batch
// by transform length, and launches it on the next of several streams, so a
// micro-batch formed from later arrivals runs while earlier ones are still on
// the device. Scratch comes from a dedicated stream-ordered memory pool and is
// returned in stream order after the batch's last kernel. When a batch's event
// completes, the worker reads its rounding margins, recomputes any block over
// the guard one mode wider, and publishes per-ticket results with submit,
// admit and completion timestamps (pa_poll / pa_wait).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "pa.h"
#include "pa_blocks.h"
#include "pa_internal.h"
#include "pa_kernels.cuh"
#include "pa_launch.h"

using namespace pa;
using pa::blocks::ClassRun;

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t ticket = 0;
    pa_block_desc_t d{};
    uint64_t L = 0;  // transform length of the block's class
    size_t bytes = 0;
    uint64_t t_submit = 0, t_admit = 0;
};

struct Slot {  // one stream and its in-flight micro-batch
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Request> reqs;
    size_t bytes = 0;
    BlockDev *h_desc = nullptr;  // pinned staging, cap entries
    float *h_marg = nullptr;     // pinned, cap entries
    uint32_t cap = 0;
    int launch_rc = PA_OK;
};

struct Twiddles {
    void *hi = nullptr, *lo = nullptr, *fine = nullptr;
    uint32_t B = 0;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct pa_server {
    pa_server_cfg_t cfg{};
    int device = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work;  // new submissions / stop
    std::condition_variable cv_done;  // completions
    std::deque<Request> queue;
    std::unordered_set<uint64_t> pending;  // queued or in flight
    std::unordered_map<uint64_t, pa_result_t> results;
    uint64_t next_ticket = 1;
    size_t inflight_bytes = 0;
    bool stop = false;
    pa_server_stats_t stats{};
    // worker-owned
    std::vector<Slot> slots;
    size_t next_slot = 0;
    cudaMemPool_t pool = nullptr;
    std::map<std::pair<uint64_t, uint32_t>, Twiddles> tw;  // by (L, F)
    std::map<std::pair<uint64_t, uint64_t>, pa_plan_t *> esc;
    cudaStream_t esc_stream = nullptr;
};

namespace {

int twiddles_for(pa_server_t *s, const Geometry &g, Twiddles *out) {
    const auto key = std::make_pair(g.L, g.F());
    auto it = s->tw.find(key);
    if (it != s->tw.end()) {
        *out = it->second;
        return PA_OK;
    }
    Twiddles t;
    int rc = pa_internal_twiddles(g.L, g.F(), (int)s->cfg.dtype, &t.hi, &t.lo, &t.B, &t.fine);
    if (rc != PA_OK) return rc;
    s->tw[key] = t;
    *out = t;
    return PA_OK;
}

// Launch one admitted micro-batch on its slot's stream (worker thread).
int launch_batch(pa_server_t *s, Slot &sl) {
    const uint32_t nb = (uint32_t)sl.reqs.size();
    const size_t esz = s->cfg.dtype == PA_FP32_GUARD ? sizeof(float2) : sizeof(double2);
    std::map<uint64_t, std::vector<uint32_t>> byL;
    for (uint32_t i = 0; i < nb; ++i) byL[sl.reqs[i].L].push_back(i);
    // one pool allocation per micro-batch: counters, descriptors, then per-class work slots
    size_t off_cnt = 0;
    size_t off_desc = align256(2 * (size_t)nb * sizeof(uint32_t));
    size_t total = off_desc + align256((size_t)nb * sizeof(BlockDev));
    std::vector<std::pair<size_t, size_t>> work_off;  // (Wf, Wi) offsets per class
    for (auto &kv : byL) {
        const size_t L = (size_t)kv.first;
        const size_t k = kv.second.size();
        const size_t wf = total;
        total += align256(k * L * esz);
        const size_t wi = total;
        total += align256(((k + 1) / 2) * L * esz);
        work_off.push_back({wf, wi});
    }
    unsigned char *mem = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&mem, total, s->pool, sl.st);
    if (e != cudaSuccess) return pa_internal_cuda_fail(e, "cudaMallocFromPoolAsync");
    uint32_t *popc = reinterpret_cast<uint32_t *>(mem + off_cnt);
    uint32_t *marg = popc + nb;
    BlockDev *d_desc = reinterpret_cast<BlockDev *>(mem + off_desc);
    // descriptors in class order; BlockDev::id = position in the micro-batch
    uint32_t pos = 0;
    std::vector<uint32_t> class_first;
    for (auto &kv : byL) {
        class_first.push_back(pos);
        for (uint32_t i : kv.second) {
            const pa_block_desc_t &d = sl.reqs[i].d;
            sl.h_desc[pos++] = BlockDev{d.n, d.m, d.key, d.seed, d.out, i, 0u};
        }
    }
    int rc = PA_OK;
    e = cudaMemcpyAsync(d_desc, sl.h_desc, nb * sizeof(BlockDev), cudaMemcpyHostToDevice, sl.st);
    if (e != cudaSuccess) rc = pa_internal_cuda_fail(e, "cudaMemcpyAsync(descriptors)");
    size_t ci = 0;
    for (auto &kv : byL) {
        if (rc != PA_OK) break;
        ClassRun c;
        if (!pa::blocks::cached_split(kv.first, s->cfg.dtype, &c.geo)) c.geo = pa::blocks::default_split(kv.first, s->cfg.dtype);
        Twiddles t;
        rc = twiddles_for(s, c.geo, &t);
        if (rc != PA_OK) break;
        c.d_blocks = d_desc + class_first[ci];
        c.nb = (uint32_t)kv.second.size();
        c.Wf = mem + work_off[ci].first;
        c.Wi = mem + work_off[ci].second;
        c.tw_hi = t.hi;
        c.tw_lo = t.lo;
        c.B = t.B;
        c.tw_fine = t.fine;
        rc = pa::blocks::run_complex(s->cfg.dtype, c, popc, marg, sl.st);
        ++ci;
    }
    if (rc == PA_OK) {
        e = cudaMemcpyAsync(sl.h_marg, marg, nb * sizeof(float), cudaMemcpyDeviceToHost, sl.st);
        if (e != cudaSuccess) rc = pa_internal_cuda_fail(e, "cudaMemcpyAsync(margins)");
    }
    cudaFreeAsync(mem, sl.st);  // stream-ordered: after the batch's last kernel
    e = cudaEventRecord(sl.done, sl.st);
    if (rc == PA_OK && e != cudaSuccess) rc = pa_internal_cuda_fail(e, "cudaEventRecord");
    return rc;
}

// Recompute one block in the next wider mode (worker thread, synchronous).
int escalate(pa_server_t *s, const pa_block_desc_t &b, float *margin, int32_t *mode) {
    const pa_dtype_t wider = s->cfg.dtype == PA_FP32_GUARD ? PA_FP64 : PA_NTT64;
    auto key = std::make_pair(b.n, b.m);
    pa_plan_t *pl = nullptr;
    auto it = s->esc.find(key);
    if (it == s->esc.end()) {
        int rc = pa_plan(b.n, b.m, wider, &pl);
        if (rc != PA_OK) return rc;
        s->esc[key] = pl;
    } else {
        pl = it->second;
    }
    pa_stream_t st = reinterpret_cast<pa_stream_t>(s->esc_stream);
    int rc = pa_set_seed(pl, b.seed, b.n + b.m - 1, st);
    if (rc != PA_OK) return rc;
    pa_batch_info_t info{margin, mode, 0, 0};
    return pa_hash_batch(pl, b.key, 1, (b.n + 63) / 64, b.out, (b.m + 63) / 64, st, &info);
}

void finish_batch(pa_server_t *s, Slot &sl) {
    const uint32_t nb = (uint32_t)sl.reqs.size();
    cudaError_t e = cudaEventSynchronize(sl.done);  // already complete when called from the poll
    int batch_rc = sl.launch_rc;
    if (batch_rc == PA_OK && e != cudaSuccess) batch_rc = pa_internal_cuda_fail(e, "batch");
    std::vector<pa_result_t> res(nb);
    uint32_t escalated = 0;
    for (uint32_t i = 0; i < nb; ++i) {
        pa_result_t &r = res[i];
        std::memset(&r, 0, sizeof(r));
        r.status = batch_rc;
        r.mode = (int32_t)s->cfg.dtype;
        r.margin = batch_rc == PA_OK ? sl.h_marg[i] : 1.f;
        if (batch_rc == PA_OK && !(r.margin <= s->cfg.guard)) {
            float m2 = 0.f;
            int32_t md = 0;
            r.status = escalate(s, sl.reqs[i].d, &m2, &md);
            r.margin = m2;
            r.mode = md;
            ++escalated;
        }
        r.t_submit_ns = sl.reqs[i].t_submit;
        r.t_admit_ns = sl.reqs[i].t_admit;
    }
    const uint64_t t = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (uint32_t i = 0; i < nb; ++i) {
            res[i].t_done_ns = t;
            s->results[sl.reqs[i].ticket] = res[i];
            s->pending.erase(sl.reqs[i].ticket);
        }
        s->inflight_bytes -= sl.bytes;
        s->stats.completed += nb;
        s->stats.escalated += escalated;
        s->stats.inflight_bytes = s->inflight_bytes;
    }
    s->cv_done.notify_all();
    sl.reqs.clear();
    sl.bytes = 0;
    sl.busy = false;
}

void worker_main(pa_server_t *s) {
    cudaSetDevice(s->device);
    for (;;) {
        // completions
        bool any_busy = false;
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            if (cudaEventQuery(sl.done) == cudaSuccess || sl.launch_rc != PA_OK) {
                finish_batch(s, sl);
            } else {
                any_busy = true;
            }
        }
        // admission into a free slot
        Slot *free_slot = nullptr;
        for (size_t k = 0; k < s->slots.size(); ++k) {
            Slot &sl = s->slots[(s->next_slot + k) % s->slots.size()];
            if (!sl.busy) {
                free_slot = &sl;
                s->next_slot = (s->next_slot + k + 1) % s->slots.size();
                break;
            }
        }
        std::vector<Request> batch;
        size_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->queue.empty() && !any_busy) break;
            if (free_slot) {
                const uint64_t t = now_ns();
                while (!s->queue.empty() && batch.size() < free_slot->cap) {
                    Request &r = s->queue.front();
                    if (s->inflight_bytes + bytes + r.bytes > s->cfg.hbm_cap_bytes) break;  // FIFO admission
                    r.t_admit = t;
                    bytes += r.bytes;
                    batch.push_back(r);
                    s->queue.pop_front();
                }
                if (!batch.empty()) {
                    s->inflight_bytes += bytes;
                    s->stats.admitted += batch.size();
                    s->stats.batches += 1;
                    s->stats.inflight_bytes = s->inflight_bytes;
                    if (s->inflight_bytes > s->stats.peak_inflight_bytes) s->stats.peak_inflight_bytes = s->inflight_bytes;
                }
            }
            if (batch.empty()) {
                if (!any_busy) {
                    // idle: sleep until a submission (or stop)
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                } else {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                }
                continue;
            }
        }
        free_slot->reqs = std::move(batch);
        free_slot->bytes = bytes;
        free_slot->busy = true;
        free_slot->launch_rc = launch_batch(s, *free_slot);
    }
}

void free_server(pa_server_t *s) {
    for (Slot &sl : s->slots) {
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
        if (sl.h_marg) cudaFreeHost(sl.h_marg);
    }
    for (auto &kv : s->tw) {
        cudaFree(kv.second.hi);
        cudaFree(kv.second.lo);
        cudaFree(kv.second.fine);
    }
    for (auto &kv : s->esc) pa_plan_destroy(kv.second);
    if (s->esc_stream) cudaStreamDestroy(s->esc_stream);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

}  // namespace

extern "C" {

int pa_server_create(const pa_server_cfg_t *cfg, pa_server_t **out) {
    if (!out) return PA_EINVAL;
    *out = nullptr;
    pa_server_cfg_t c{};
    if (cfg) c = *cfg;
    if (c.hbm_cap_bytes == 0) c.hbm_cap_bytes = 40ull * 1000 * 1000 * 1000;
    if (c.max_queue == 0) c.max_queue = 65536;
    if (c.max_batch == 0) c.max_batch = 64;
    if (c.streams == 0) c.streams = 4;
    if (!(c.guard > 0.f)) c.guard = 0.25f;
    if (c.dtype != PA_FP32_GUARD && c.dtype != PA_FP64) return PA_EINVAL;
    if (c.streams > 64 || c.max_batch > 65536) return PA_EINVAL;
    pa_server_t *s = new pa_server_t();
    s->cfg = c;
    cudaGetDevice(&s->device);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    cudaError_t e = cudaMemPoolCreate(&s->pool, &props);
    if (e != cudaSuccess) {
        free_server(s);
        return pa_internal_cuda_fail(e, "cudaMemPoolCreate");
    }
    uint64_t thr = c.hbm_cap_bytes;  // keep up to the cap resident between batches
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    s->slots.resize(c.streams);
    for (Slot &sl : s->slots) {
        sl.cap = c.max_batch;
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.h_desc, c.max_batch * sizeof(BlockDev)) != cudaSuccess ||
            cudaMallocHost(&sl.h_marg, c.max_batch * sizeof(float)) != cudaSuccess) {
            free_server(s);
            return PA_ENOMEM;
        }
    }
    if (cudaStreamCreateWithFlags(&s->esc_stream, cudaStreamNonBlocking) != cudaSuccess) {
        free_server(s);
        return PA_ECUDA;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return PA_OK;
}

int pa_submit(pa_server_t *s, const pa_block_desc_t *b, uint64_t *ticket) {
    if (!s || !b || !ticket) return PA_EINVAL;
    if (b->n == 0 || b->m == 0 || b->m > b->n || b->n > (1ull << 27) || !b->key || !b->seed || !b->out) return PA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(b->key) | reinterpret_cast<uintptr_t>(b->seed) |
         reinterpret_cast<uintptr_t>(b->out)) & 15u)
        return PA_EINVAL;
    Request r;
    r.d = *b;
    r.L = pa::blocks::class_length(b->n, b->m, s->cfg.dtype);
    if (r.L == 0) return PA_EUNSUPPORTED;
    r.bytes = pa::blocks::scratch_per_block(r.L, s->cfg.dtype);
    if (r.bytes > s->cfg.hbm_cap_bytes) return PA_EINVAL;  // could never be admitted
    r.t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return PA_EINVAL;
        if (s->pending.size() >= s->cfg.max_queue) {
            s->stats.rejected += 1;
            return PA_EAGAIN;
        }
        r.ticket = s->next_ticket++;
        s->queue.push_back(r);
        s->pending.insert(r.ticket);
        s->stats.submitted += 1;
        *ticket = r.ticket;
    }
    s->cv_work.notify_one();
    return PA_OK;
}

int pa_poll(pa_server_t *s, uint64_t ticket, pa_result_t *result) {
    if (!s || !result) return PA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it != s->results.end()) {
        *result = it->second;
        s->results.erase(it);
        return PA_OK;
    }
    return s->pending.count(ticket) ? PA_EPENDING : PA_EINVAL;
}

int pa_wait(pa_server_t *s, uint64_t ticket, uint32_t timeout_ms, pa_result_t *result) {
    if (!s || !result) return PA_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = s->results.find(ticket);
        if (it != s->results.end()) {
            *result = it->second;
            s->results.erase(it);
            return PA_OK;
        }
        if (!s->pending.count(ticket)) return PA_EINVAL;
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !s->results.count(ticket))
            return PA_ETIMEOUT;
    }
}

int pa_server_stats(pa_server_t *s, pa_server_stats_t *out) {
    if (!s || !out) return PA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = s->queue.size();
    return PA_OK;
}

int pa_server_destroy(pa_server_t *s) {
    if (!s) return PA_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaDeviceSynchronize();
    free_server(s);
    return PA_OK;
}

}  // extern "C"

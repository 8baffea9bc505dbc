/*
 * pa.h -- C ABI of the GB300 Toeplitz-hash privacy-amplification library (libpa.so).
 *
 * The library computes the privacy-amplification hash of the paper's Section 2.2:
 * an m x n binary Toeplitz matrix T, fixed by an (n+m-1)-bit seed s, compresses an
 * n-bit reconciled key x into the m-bit final key
 *
 *     y = T x mod 2,   T[i][j] = s[i - j + n - 1]   (0 <= i < m, 0 <= j < n),
 *
 * evaluated, as in Eq. 4, as a linear convolution of s and x through a cyclic
 * convolution of length L >= n+m-1 computed with FFTs (forward transform,
 * pointwise product with the seed's spectrum, inverse transform, rounding,
 * mod 2). All arithmetic runs in the library's own CUDA kernels on one GPU.
 *
 * Bit layout (every bit-vector argument): bit j is bit (j % 64) of 64-bit word
 * j / 64, little-endian words. A key occupies ceil(n/64) words, a seed
 * ceil((n+m-1)/64) words, a final key ceil(m/64) words. Input bits past the
 * vector's length are ignored; output bits at positions >= m are written as 0.
 *
 * Errors: every entry point returns an int, PA_OK (0) on success or one of the
 * negative PA_E* codes below; pa_strerror() names them. No C++ exception crosses
 * this boundary. Device pointers must be 16-byte aligned.
 *
 * Environment (read when a plan or batch is built; all optional):
 *   PA_PLAN_TUNE=0    take the default pass split instead of timing every split
 *   PA_TUNE_CACHE     file that keeps the uneven batches' tuned splits across processes
 *   PA_WORK_BYTES     work-buffer budget of one launch chunk in bytes (default 4 GiB): a
 *                     batch whose key pairs need more runs in several chunks
 *   PA_POW2_ONLY      (any value) restrict transform lengths to powers of two
 *   PA_STATIC_GUARD   rounding-margin threshold of pa_hash_static's guard (default 0.25;
 *                     read at every call; a negative value forces its escalation path)
 *
 * Threads: a plan may be used from one host thread at a time. Its calls may take
 * different streams: each batch or seed upload first waits (on the device) for the
 * plan's previous one, so the calls on one plan run in issue order whatever
 * stream carries them, while different plans on different streams overlap.
 * A server is thread-safe.
 */
#ifndef PA_H_
#define PA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle (the same object as cudaStream_t); NULL is the legacy default stream. */
typedef struct CUstream_st *pa_stream_t;

/* Error codes. */
#define PA_OK 0
#define PA_EINVAL (-1)       /* bad size, null or misaligned pointer, seed length mismatch, bad handle */
#define PA_ENOMEM (-2)       /* device or pinned-host allocation failed */
#define PA_EAGAIN (-3)       /* server: admission cap reached and queue full, retry later */
#define PA_EPENDING (-4)     /* server: the ticket has not completed yet */
#define PA_ETIMEOUT (-5)     /* a bounded wait expired */
#define PA_EPRECISION (-6)   /* no precision mode produced an unambiguous rounding (should not happen) */
#define PA_ECUDA (-7)        /* a CUDA runtime call failed; see pa_last_cuda_error() */
#define PA_ENOSEED (-8)      /* pa_hash_batch before pa_set_seed */
#define PA_EUNSUPPORTED (-9) /* size or mode this build does not handle */

/*
 * Arithmetic of the transform (paper Section 5 names the precision of the FFT
 * as the open question; these are the three answers the library offers).
 *   PA_FP64        double-precision complex FFTs.
 *   PA_FP32_GUARD  single-precision complex FFTs; every key's rounding margin
 *                  max_i |v_i - rint(v_i)| is checked, and a key whose margin
 *                  exceeds 0.25 is recomputed in FP64.
 *   PA_NTT64       exact number-theoretic transform modulo p = 2^64 - 2^32 + 1.
 * The output bits are the same in every mode.
 */
typedef enum { PA_FP64 = 0, PA_FP32_GUARD = 1, PA_NTT64 = 2 } pa_dtype_t;

typedef struct pa_plan pa_plan_t;

/* Per-key diagnostics filled by pa_hash_batch when the caller passes one. */
typedef struct {
    float *margin;       /* host array of nkeys, or NULL: rounding margin of the mode that produced each key */
    int32_t *mode;       /* host array of nkeys, or NULL: the pa_dtype_t that produced each key */
    uint32_t escalated;  /* out: number of keys recomputed in a wider mode */
    uint32_t reserved;
} pa_batch_info_t;

/*
 * pa_plan -- choose the transform for keys of n bits hashed to m bits.
 * Paper Section 2.2 (FFT length n+r-1 for the standard Toeplitz matrix) and
 * Algorithm 1 (a long FFT split into passes of short FFTs): the plan picks the
 * smallest complex length L >= max(n+m-1, 4096) of the form ro * 2^k with ro in
 * {1, 3, 5, 9} (ro = 1 only for PA_NTT64), factors it into two or three passes,
 * builds twiddle tables, and allocates the seed-spectrum slot (L complex values)
 * on the current CUDA device. Where L has several valid pass splits, the first
 * plan of each (L, dtype) in a process times every split on a batch of zero keys
 * (stream-ordered on a private stream, up to 32 key pairs; set the environment
 * variable PA_PLAN_TUNE=0 to skip this and take the default split) and later
 * plans reuse the winner. Work buffers are allocated by the first pa_hash_batch
 * that needs them and kept until pa_plan_destroy.
 *   n      key length in bits, 1 <= n <= 2^27
 *   m      final-key length in bits, 1 <= m <= n
 *   dtype  arithmetic of the transform (see pa_dtype_t)
 *   out    receives the plan; owned by the caller, released with pa_plan_destroy
 * Returns PA_EINVAL for bad sizes, PA_ENOMEM, PA_EUNSUPPORTED, PA_ECUDA.
 */
int pa_plan(uint64_t n, uint64_t m, pa_dtype_t dtype, pa_plan_t **out);

/*
 * pa_plan_splits -- the pass splits pa_plan chooses among for (n, m, dtype) (no GPU work).
 * Writes up to `cap` entries (L1[i], L2[i], L3[i]) in the convention of pa_plan_shape and
 * the total number of splits to *count. Every split computes the same bits.
 * Returns PA_EINVAL for bad arguments, PA_EUNSUPPORTED if no length is supported.
 */
int pa_plan_splits(uint64_t n, uint64_t m, pa_dtype_t dtype, uint32_t *L1, uint32_t *L2, uint32_t *L3, int cap,
                   int *count);

/*
 * pa_plan_split -- pa_plan with the pass split fixed to (L1, L2, L3), one of the splits
 * pa_plan_splits lists (PA_EINVAL otherwise). No timing is done.
 */
int pa_plan_split(uint64_t n, uint64_t m, pa_dtype_t dtype, uint32_t L1, uint32_t L2, uint32_t L3, pa_plan_t **out);

/*
 * Security parameter of the hash (paper Section 2.1, Eq. 1). If Eve holds at most t
 * bits of information about the n-bit reconciled key, hashing it to r bits with a
 * universal (Toeplitz) hash leaves her I(K; g, V) <= 2^-s / ln 2 bits about the
 * final key, with security coefficient s = n - t - r.
 * pa_final_key_length: r = n - t - s for a wanted s; PA_EINVAL unless r >= 1
 *   (t < n and s < n - t). Host only.
 * pa_leakage_bound: the right-hand side 2^-(n-t-r) / ln 2 of Eq. 1 (for n - t - r <= 0
 *   the value is >= 1/ln 2, i.e. no guarantee). Host only.
 */
int pa_final_key_length(uint64_t n, uint64_t t, uint64_t s, uint64_t *r);
double pa_leakage_bound(uint64_t n, uint64_t t, uint64_t r);

/*
 * pa_plan_modified -- plan for the modified Toeplitz hash of Section 2.2 (Eq. 2-3):
 * the m x n matrix [I_m, T'] with T' the m x (n-m) Toeplitz block
 * T'[i][j] = s[i - j + n - m - 1] of an (n-1)-bit seed s, so that
 *     y_i = x_i XOR (XOR_{j < n-m} s[i - j + n - m - 1] AND x_{m+j}),   0 <= i < m.
 * (The paper prints the block as V_{r-1-i+j}: the same map with the seed reversed.)
 * The transform length only has to cover n-1 instead of n+m-1. Use the plan with
 * pa_set_seed (seed_bits = n - 1), pa_hash_batch / pa_hash_host and their async
 * forms exactly as a pa_plan plan; keys are n bits. 1 <= m < n <= 2^27.
 */
int pa_plan_modified(uint64_t n, uint64_t m, pa_dtype_t dtype, pa_plan_t **out);

/* Release a plan and all device memory it owns. NULL is accepted. Synchronizes the device. */
int pa_plan_destroy(pa_plan_t *plan);

/*
 * pa_set_seed -- cache the spectrum of the Toeplitz seed (Eq. 4: FFT(V_n),
 * computed once and reused by every key hashed with this seed).
 *   seed_dev   device pointer, ceil(seed_bits/64) words, caller-owned, read during
 *              the call only (stream-ordered)
 *   seed_bits  must equal n+m-1 (PA_EINVAL otherwise)
 *   stream     CUDA stream the transform is issued on; asynchronous
 */
int pa_set_seed(pa_plan_t *plan, const uint64_t *seed_dev, uint64_t seed_bits, pa_stream_t stream);

/*
 * pa_hash_batch -- y_k = T x_k mod 2 for nkeys keys that share the plan's seed
 * (Eq. 3-4 for every key; two keys ride in one complex transform as its real
 * and imaginary parts, the idea of Eq. 5-10 applied to two keys). A batch of
 * one key in PA_FP32_GUARD or PA_FP64 runs in a transform of half the length,
 * its even and odd bits as the real and imaginary parts (Eq. 5-10's split of a
 * complex transform into two real ones, applied per bin pair).
 *   keys_dev          device pointer; key k starts at keys_dev + k*key_stride_words
 *   nkeys             number of keys, >= 1
 *   key_stride_words  >= ceil(n/64), even (16-byte alignment of every key)
 *   out_dev           device pointer; final key k starts at out_dev + k*out_stride_words
 *   out_stride_words  >= ceil(m/64), even
 *   stream            CUDA stream; kernels are issued asynchronously on it
 *   info              optional per-key diagnostics (may be NULL)
 * Synchronization: in PA_FP32_GUARD mode, and in any mode when info != NULL, the
 * call waits for the stream to read the rounding margins back (the guard of
 * Section 5's precision question needs them on the host); otherwise it returns
 * after issuing the kernels. Returns PA_ENOSEED if no seed was set.
 * Device waits are bounded: the fused convolution kernel waits on its own
 * asynchronous copies for at most 1 s. If a wait runs out, the plan's device
 * error word is set and the next call that synchronizes (this one in
 * PA_FP32_GUARD mode or with info) returns PA_ETIMEOUT, clears the word, and the
 * outputs of the batches since the last synchronizing call are not valid.
 */
int pa_hash_batch(pa_plan_t *plan, const uint64_t *keys_dev, uint32_t nkeys, uint64_t key_stride_words,
                  uint64_t *out_dev, uint64_t out_stride_words, pa_stream_t stream, pa_batch_info_t *info);

/*
 * pa_hash_batch_async / pa_batch_finish -- pa_hash_batch in two halves, so that a
 * host thread can issue batches of several plans back to back and run the
 * guard of each afterwards (no idle GPU between batches).
 * pa_hash_batch_async checks the arguments as pa_hash_batch does, issues the
 * kernels and the read-back of the rounding margins on the stream, and returns.
 * pa_batch_finish waits for that read-back, recomputes every key whose margin
 * fails the guard one mode wider (as pa_hash_batch does) and fills info (may be
 * NULL). The outputs are final once pa_batch_finish has returned PA_OK. Between
 * the two calls the plan accepts no other hash call (PA_EAGAIN); pa_batch_finish
 * without an issued batch returns PA_EINVAL. pa_hash_batch is
 * pa_hash_batch_async followed by pa_batch_finish (the latter skipped in
 * PA_FP64 / PA_NTT64 mode without info).
 */
int pa_hash_batch_async(pa_plan_t *plan, const uint64_t *keys_dev, uint32_t nkeys, uint64_t key_stride_words,
                        uint64_t *out_dev, uint64_t out_stride_words, pa_stream_t stream);
int pa_batch_finish(pa_plan_t *plan, pa_batch_info_t *info);

/*
 * pa_hash_host_async / pa_hash_host -- key ingestion and final-key egress around the
 * hash (the QKD pipeline hands raw keys over in host memory and takes final keys
 * back, the paper's Fig. 1): keys are copied from host memory into plan-owned
 * device rows on a copy stream, hashed on `stream`, and the final keys copied back
 * to host memory on a second copy stream, so consecutive batches (of this and of
 * other plans) overlap their copies with each other's compute. The copies overlap
 * only from pinned host memory (cudaHostAlloc / cudaHostRegister); pageable memory
 * works but serialises.
 *   keys_host          host pointer; key k starts at keys_host + k*key_stride_words (>= ceil(n/64))
 *   out_host           host pointer; final key k at out_host + k*out_stride_words (>= ceil(m/64));
 *                      only the ceil(m/64) words of each row are written (tail bits zero)
 * pa_hash_host_async returns after issuing; pa_batch_finish (above) waits for the
 * read-back, runs the guard, and rewrites in host memory the rows of the keys it
 * recomputed. The host rows are final once pa_batch_finish returns PA_OK; the
 * caller keeps both host buffers alive and unmodified until then. pa_hash_host is
 * the two calls in one. Errors as pa_hash_batch (no alignment rule for host pointers).
 */
int pa_hash_host_async(pa_plan_t *plan, const uint64_t *keys_host, uint32_t nkeys, uint64_t key_stride_words,
                       uint64_t *out_host, uint64_t out_stride_words, pa_stream_t stream);
int pa_hash_host(pa_plan_t *plan, const uint64_t *keys_host, uint32_t nkeys, uint64_t key_stride_words,
                 uint64_t *out_host, uint64_t out_stride_words, pa_stream_t stream, pa_batch_info_t *info);

/*
 * pa_plan_set_guard -- rounding-margin threshold of the FP32 guard (default 0.25,
 * the value the guard is specified with). A key whose margin max_i |w_i - rint(w_i)|
 * exceeds it is recomputed in FP64. Lowering it (e.g. to -1) forces every key
 * through the escalation path; tests use that to exercise it.
 */
int pa_plan_set_guard(pa_plan_t *plan, float threshold);

/*
 * pa_plan_set_staged -- run the last pass of this plan's batches (on = 1) as a persistent
 * kernel that stages its input tiles in shared memory with tiled asynchronous copies (the
 * TMA) while it transforms the previous tile, or (on = 0, the default) as one CTA per tile
 * with plain loads. Applies to PA_FP32_GUARD plans whose first pass length is at most 256
 * (other plans ignore it). Both give the same bits. Measured on the DV-QKD batches: the
 * staged pass is about 6 % faster when one batch runs alone, but a step whose batches
 * overlap on two streams is about 2 % slower with it, because the persistent kernel holds
 * its SMs while the other stream's kernels wait. No counterpart in the paper.
 */
int pa_plan_set_staged(pa_plan_t *plan, int on);

/*
 * pa_plan_set_storage_bits -- reduced-precision storage study (the paper's Section 5 asks
 * how far the FFT's precision can go down before privacy amplification breaks). With
 * 1 <= bits <= 22, every value a PA_FP32_GUARD plan stores between its passes (the key
 * transforms after each pass, and the seed spectrum) is rounded to `bits` explicit
 * significand bits, round to nearest even, as if it were kept in a narrower format with
 * FP32's exponent range (10 bits: FP16's significand; 7: BF16's); the arithmetic inside
 * each pass stays FP32. Each rounding is one extra elementwise pass over the slots, so
 * this is a measurement mode, not a fast one. Margins grow accordingly, the guard
 * escalates every key whose margin exceeds its threshold, and the output bits stay exact.
 * bits = 23 (or 0) turns it off. The call discards the cached seed spectrum: call
 * pa_set_seed again before hashing. Batches of this plan use key pairs only (a lone key
 * does not take the half-length form). PA_EUNSUPPORTED for other modes, PA_EINVAL for
 * bits > 23. No counterpart in the paper's method itself.
 */
int pa_plan_set_storage_bits(pa_plan_t *plan, uint32_t bits);

/*
 * pa_plan_expire_waits -- test hook for the device-side wait limit (library robustness;
 * the paper has no counterpart). The staged last pass (pa_plan_set_staged) waits for each
 * of its tiled copies with a time limit;
 * when a wait runs out the kernel sets bit 0 of the plan's device error word and returns
 * instead of spinning. After this call, the next `launches` launches of that kernel issue
 * no copy and wait 10 microseconds on a barrier phase that nothing can complete, so their
 * wait runs out with no copy in flight. The batch's synchronising call (pa_hash_batch of a
 * PA_FP32_GUARD plan or with info, pa_hash_host, pa_batch_finish) then returns PA_ETIMEOUT
 * and clears the word; that batch's outputs are not valid, and the plan stays usable.
 * Every other call reports such an error only at the next synchronising call on the plan.
 * Returns PA_EUNSUPPORTED for plans whose last pass is not staged (staging off, or a plan
 * it does not apply to), PA_EINVAL for a NULL plan.
 */
int pa_plan_expire_waits(pa_plan_t *plan, uint32_t launches);

/* Plan introspection (no GPU work): transform length L and pass lengths L1, L2, L3 (L3 = 1 for two passes). */
int pa_plan_shape(const pa_plan_t *plan, uint64_t *L, uint32_t *L1, uint32_t *L2, uint32_t *L3);

/* ---------------------------------------------------------------------------------------
 * Uneven batch: blocks of different (n, m), each with its own key and seed, as reconciliation
 * emits them.
 * ------------------------------------------------------------------------------------- */

/* One privacy-amplification block. All pointers are device pointers, 16-byte aligned:
 * key ceil(n/64) words, seed ceil((n+m-1)/64) words, out ceil(m/64) words. */
typedef struct {
    uint64_t n, m;
    const uint64_t *key;
    const uint64_t *seed;
    uint64_t *out;
} pa_block_desc_t;

typedef struct pa_uneven pa_uneven_t;

/*
 * pa_uneven_create -- plan an uneven batch. Blocks are grouped by transform length L, the
 * smallest smooth length ro * 2^k >= max(n+m-1, 2^12) with ro in {1, 3, 5, 9} (PA_NTT64:
 * powers of two only), as pa_plan chooses it; every class gets its own work buffers, twiddle
 * tables and a device copy of its block descriptors, and its pass split is chosen by the
 * built-in autotuner (timed on the class's own buffers, cached per (L, dtype) for the process
 * and, if the environment variable PA_TUNE_CACHE names a file, across processes).
 * In PA_FP32_GUARD and PA_FP64 mode each block's key and seed share one complex transform,
 * z = x + i*sigma, and are separated after the forward transform with the paper's real-valued
 * FFT identities (Eq. 5-10); two blocks share each inverse transform. PA_NTT64 blocks run one
 * exact transform chain each. With use_graph != 0 all launches are captured once into a CUDA
 * graph (one branch per length class, the classes run concurrently) and pa_uneven_run replays it.
 *   blocks   caller array of nblocks descriptors (copied; the device buffers they name must
 *            stay valid until the batch is destroyed or updated)
 * Returns PA_EINVAL (bad sizes, alignment, nblocks == 0), PA_ENOMEM, PA_EUNSUPPORTED, PA_ECUDA.
 */
int pa_uneven_create(const pa_block_desc_t *blocks, uint32_t nblocks, pa_dtype_t dtype, int use_graph,
                     pa_uneven_t **out);

/*
 * pa_uneven_update -- point the batch at new key/seed/output buffers. Block i must keep the
 * (n, m) it was created with (PA_EINVAL otherwise). Stream-ordered on `stream`.
 */
int pa_uneven_update(pa_uneven_t *batch, const pa_block_desc_t *blocks, uint32_t nblocks, pa_stream_t stream);

/*
 * pa_uneven_run -- hash every block (graph replay or direct launches on `stream`). In
 * PA_FP32_GUARD mode, or when info != NULL, waits for the per-block margins and recomputes
 * blocks over the 0.25 guard in FP64 (then NTT64); info->margin / info->mode are indexed by
 * block.
 */
int pa_uneven_run(pa_uneven_t *batch, pa_stream_t stream, pa_batch_info_t *info);

/* Rounding-margin threshold of the batch's guard (default 0.25); see pa_plan_set_guard. */
int pa_uneven_set_guard(pa_uneven_t *batch, float threshold);

/* Release the batch and its device memory (synchronizes the device). NULL is accepted. */
int pa_uneven_destroy(pa_uneven_t *batch);

/* Describe the split chosen for one length class: returns the number of classes in *nclasses
 * and, for class c < nclasses, its L, pass lengths and number of blocks. */
int pa_uneven_class(const pa_uneven_t *batch, uint32_t c, uint32_t *nclasses, uint64_t *L, uint32_t *L1,
                    uint32_t *L2, uint32_t *L3, uint32_t *nblocks);

/* One-shot convenience: create (without a graph), run, destroy. */
int pa_hash_uneven(const pa_block_desc_t *blocks, uint32_t nblocks, pa_dtype_t dtype, pa_stream_t stream,
                   pa_batch_info_t *info);

/* ---------------------------------------------------------------------------------------
 * Serving loop: continuous batching of blocks submitted one at a time.
 * ------------------------------------------------------------------------------------- */

typedef struct pa_server pa_server_t;

typedef struct {
    uint64_t hbm_cap_bytes;  /* admission cap on the device scratch of in-flight blocks (0: 40e9) */
    pa_dtype_t dtype;        /* PA_FP32_GUARD or PA_FP64 (a zeroed struct selects PA_FP64) */
    uint32_t max_queue;      /* queued + in-flight blocks before pa_submit returns PA_EAGAIN (0: 65536) */
    uint32_t max_batch;      /* blocks admitted into one micro-batch (0: 64) */
    uint32_t streams;        /* micro-batches in flight at once, one stream each (0: 4) */
    float guard;             /* rounding-margin threshold (<= 0: 0.25) */
} pa_server_cfg_t;

typedef struct {
    int32_t status;        /* PA_OK, or the error that ended this block */
    int32_t mode;          /* pa_dtype_t that produced the bits */
    float margin;          /* rounding margin of that mode */
    uint32_t reserved;
    uint64_t t_submit_ns;  /* steady-clock timestamps: pa_submit, admission, completion seen by the server */
    uint64_t t_admit_ns;
    uint64_t t_done_ns;
} pa_result_t;

typedef struct {
    uint64_t submitted, admitted, completed, escalated, rejected, batches;
    uint64_t queued;               /* waiting for admission now */
    uint64_t inflight_bytes;       /* admitted scratch now */
    uint64_t peak_inflight_bytes;  /* largest admitted scratch so far (never above the cap) */
} pa_server_stats_t;

/*
 * pa_server_create -- start a serving loop on the current device (one worker thread).
 * Blocks are admitted first-come first-served while the scratch of everything in flight
 * (about 1.5 * L * element size per block) fits under cfg->hbm_cap_bytes; each admitted
 * micro-batch is grouped by transform length and run like an uneven batch (Eq. 5-10 key+seed
 * transforms) on the next free stream, so later arrivals run while earlier ones are on the
 * device. Scratch comes from a dedicated stream-ordered memory pool. Thread-safe.
 */
int pa_server_create(const pa_server_cfg_t *cfg, pa_server_t **out);

/*
 * pa_submit -- queue one block; *ticket identifies it in pa_poll / pa_wait. The block's device
 * buffers must stay valid until its result has been collected. Returns PA_EAGAIN when
 * cfg->max_queue blocks are already queued or in flight, PA_EINVAL for bad descriptors or a
 * block whose scratch alone exceeds the cap.
 */
int pa_submit(pa_server_t *server, const pa_block_desc_t *block, uint64_t *ticket);

/* Non-blocking: PA_OK and *result when the ticket has completed (the ticket is then released),
 * PA_EPENDING while it is queued or running, PA_EINVAL for an unknown or released ticket. */
int pa_poll(pa_server_t *server, uint64_t ticket, pa_result_t *result);

/* Blocking variant of pa_poll with a bound: PA_ETIMEOUT after timeout_ms. */
int pa_wait(pa_server_t *server, uint64_t ticket, uint32_t timeout_ms, pa_result_t *result);

int pa_server_stats(pa_server_t *server, pa_server_stats_t *stats);

/* Finish every queued block, stop the worker and release the server. NULL is accepted. */
int pa_server_destroy(pa_server_t *server);

/*
 * Kernel timing (measurement support, no counterpart in the paper). When enabled,
 * every kernel launch of the plan is bracketed by CUDA events recorded on the
 * launching stream. pa_profile_read waits for the recorded events, adds their
 * elapsed times to per-kernel totals and returns them; reset != 0 clears the totals.
 */
typedef struct {
    const char *name;      /* kernel family: "prep", "fwd_keys", "fwd_seed", "mid_fwd", "middle_conv", ... */
    uint64_t launches;     /* launches since the last reset */
    double total_ms;       /* summed event time */
} pa_kernel_stat_t;

#define PA_NUM_KERNEL_KINDS 8

int pa_profile_enable(pa_plan_t *plan, int enable);
/* stats: caller array of PA_NUM_KERNEL_KINDS entries; *count receives the number filled. */
int pa_profile_read(pa_plan_t *plan, pa_kernel_stat_t *stats, int *count, int reset);

/*
 * pa_alu_peaks -- measured arithmetic peaks of the current device for the rooflines of
 * the FP64 and exact modes (measurement support; the paper has no counterpart): the rate
 * of independent double-precision fused multiply-adds in GFLOP/s (2 flops each), and the
 * rate of products modulo p = 2^64 - 2^32 + 1 (64 x 64 -> 128-bit multiply and the
 * reduction the NTT64 transform uses) in G products/s. Runs two short kernels on
 * `stream` (a few ms), timed with CUDA events, and waits for them. Both outputs are host
 * pointers. Returns PA_EINVAL for NULL outputs, PA_ECUDA on a CUDA error.
 */
int pa_alu_peaks(double *fp64_gflops, double *zp_gmul_s, pa_stream_t stream);

/*
 * pa_hash_static -- the hash of one or two keys that share one seed, computed
 * without allocating any memory. The paper has no counterpart to this entry
 * point: it serves callers that cannot call cudaMalloc, such as a process whose
 * device memory is wholly reserved by another framework's caching allocator, a
 * real-time key-distillation loop that must not pay cudaMalloc's latency or
 * cudaFree's device-wide synchronisation, or an embedding that forbids dynamic
 * allocation after start-up.
 *
 * All scratch (work slot, seed spectrum, twiddle tables, per-key counters) sits
 * in one static device array of 65 MiB inside libpa.so, which every GPU that
 * loads the library holds until the process exits. Limits: n + m - 1 <= 2^21
 * (larger sizes return PA_EUNSUPPORTED), nkeys is 1 or 2. Arguments are those of
 * pa_plan + pa_set_seed + pa_hash_batch for one call (seed_dev holds n+m-1 bits);
 * margin, if not NULL, receives the larger rounding margin of the keys (host).
 *
 * The first call on a device looks up the array's device address on that device
 * (cudaGetSymbolAddress) and keeps it for that device's context; a call after the
 * context was reset (cudaDeviceReset) looks it up again. Make the first call on a
 * device, and the first after a reset, before any stream capture. Every
 * call re-transforms the seed and reuses the same array, which keeps the last
 * call's contents: calls that overlap on the GPU (different streams, or threads)
 * race and must be serialised by the caller. PA_FP32_GUARD calls, and any call
 * with margin != NULL, wait for the stream to read the margin back; a key pair
 * whose margin exceeds 0.25 is recomputed in FP64 (then NTT64) in the same array.
 */
int pa_hash_static(uint64_t n, uint64_t m, pa_dtype_t dtype, const uint64_t *seed_dev, const uint64_t *keys_dev,
                   uint32_t nkeys, uint64_t key_stride_words, uint64_t *out_dev, uint64_t out_stride_words,
                   pa_stream_t stream, float *margin);

/* Text for an error code; never NULL. */
const char *pa_strerror(int code);

/* The last CUDA runtime error string seen by this thread ("" if none). */
const char *pa_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PA_H_ */

/*
 * pa_oracle.c -- CPU oracle for Toeplitz-hash privacy amplification.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product path
 * (the CUDA library and its Python binding) never calls it, and the two
 * share no code.
 *
 * What it computes (paper Section 2.2, the standard Toeplitz hash, and
 * Eq. 3-4, which write the hash as a matrix-vector product over GF(2)):
 * an m x n binary Toeplitz matrix T is fixed by an (n+m-1)-bit seed s and
 * the final key is y = T x mod 2. The FFT of Eq. 4 is only a faster route
 * to the same product, so the oracle is the product's plain definition:
 *
 *     y_i = XOR_{0 <= j < n}  s[i - j + n - 1] AND x[j],   0 <= i < m,
 *
 * i.e. T[i][j] = s[i - j + n - 1] (constant along diagonals i - j). Entry
 * T[0][n-1] = s[0] and T[m-1][0] = s[n+m-2], so the seed holds exactly the
 * n+m-1 random bits of Section 2.2.
 *
 * Algorithm (direct O(n m) bit-parallel product, the classical scheme the
 * paper compares against in Section 1 and Table 3): with the reversed key
 * xr[j'] = x[n-1-j'] the row sum becomes sum_{j'} s[i + j'] xr[j'], so row
 * i is the parity of popcount(s[i .. i+n-1] AND xr), evaluated 64 bits at a
 * time. Rows are independent and are split across POSIX threads.
 *
 * The definition holds for any n, m >= 1 (a tall block, m > n, reads the same
 * n+m-1 seed bits); the product's API limits the standard hash to m <= n, and
 * the modified Toeplitz hash of Eq. 2-3 uses blocks with m > n.
 *
 * Packed layout: bit j of a bit-vector is bit (j % 64) of 64-bit word j/64.
 * Key bits at positions >= n and seed bits at positions >= n+m-1 are
 * ignored; output bits at positions >= m are written as zero.
 *
 * Portable C11: no SIMD intrinsics, no inline assembly.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

static inline uint64_t nwords(uint64_t bits) { return (bits + 63) / 64; }

static inline int get_bit(const uint64_t *v, uint64_t j) { return (int)((v[j >> 6] >> (j & 63)) & 1u); }

static inline unsigned popcount64(uint64_t w) { return (unsigned)__builtin_popcountll(w); }

/* 64 bits of v starting at bit position pos; bits past nbits read as zero. */
static uint64_t window64(const uint64_t *v, uint64_t nbits, uint64_t pos) {
    uint64_t nw = nwords(nbits);
    uint64_t q = pos >> 6, r = pos & 63;
    uint64_t lo = (q < nw) ? v[q] : 0;
    uint64_t hi = (q + 1 < nw) ? v[q + 1] : 0;
    uint64_t w = r ? ((lo >> r) | (hi << (64 - r))) : lo;
    /* clear bits at or beyond nbits */
    if (pos >= nbits) return 0;
    if (nbits - pos < 64) w &= (((uint64_t)1) << (nbits - pos)) - 1;
    return w;
}

typedef struct {
    uint64_t n, m;
    const uint64_t *seed; /* n+m-1 bits */
    const uint64_t *xr;   /* reversed key, n bits, tail zero */
    uint64_t row0, row1;  /* rows [row0, row1) of this worker, row0 % 64 == 0 unless first */
    uint64_t *out;
} job_t;

/* y_i for one row: parity of popcount(s[i .. i+n-1] AND xr). */
static int row_parity(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *xr, uint64_t i) {
    uint64_t sbits = n + m - 1;
    uint64_t nw = nwords(n);
    uint64_t acc = 0;
    for (uint64_t w = 0; w < nw; ++w) acc += popcount64(window64(seed, sbits, i + 64 * w) & xr[w]);
    return (int)(acc & 1u);
}

static void *worker(void *arg) {
    job_t *jb = (job_t *)arg;
    for (uint64_t i = jb->row0; i < jb->row1; ++i) {
        uint64_t bit = (uint64_t)row_parity(jb->n, jb->m, jb->seed, jb->xr, i);
        uint64_t mask = ((uint64_t)1) << (i & 63);
        jb->out[i >> 6] = (jb->out[i >> 6] & ~mask) | (bit << (i & 63));
    }
    return NULL;
}

/*
 * Rows [row0, row1) of y = T x mod 2 into out (ceil(m/64) words). Bits of
 * rows outside the range are left as they are, except that when the range
 * reaches row m-1 the output bits >= m are cleared. threads <= 0 means 1.
 */
int pa_oracle_hash_rows(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key,
                        uint64_t row0, uint64_t row1, uint64_t *out, int threads) {
    if (n == 0 || m == 0 || !seed || !key || !out || row0 > row1 || row1 > m) return ORACLE_EINVAL;
    uint64_t nw = nwords(n);
    uint64_t *xr = (uint64_t *)calloc(nw ? nw : 1, sizeof(uint64_t));
    if (!xr) return ORACLE_ENOMEM;
    for (uint64_t j = 0; j < n; ++j)
        if (get_bit(key, n - 1 - j)) xr[j >> 6] |= ((uint64_t)1) << (j & 63);

    if (threads < 1) threads = 1;
    uint64_t rows = row1 - row0;
    /* chunks are multiples of 64 rows so that no two threads share an output word */
    uint64_t per = (rows + (uint64_t)threads - 1) / (uint64_t)threads;
    per = (per + 63) & ~(uint64_t)63;
    if (per == 0) per = 64;
    int nt = 0;
    job_t *jobs = (job_t *)calloc((size_t)threads, sizeof(job_t));
    pthread_t *tids = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) { free(xr); free(jobs); free(tids); return ORACLE_ENOMEM; }
    uint64_t start = row0;
    /* first chunk ends on a 64-row boundary so that all later chunks start on one */
    while (start < row1 && nt < threads) {
        uint64_t end = ((start / 64) * 64) + per;
        if (end > row1 || nt == threads - 1) end = row1;
        jobs[nt] = (job_t){n, m, seed, xr, start, end, out};
        ++nt;
        start = end;
    }
    int *ok = (int *)calloc((size_t)threads, sizeof(int));
    if (!ok) { free(xr); free(jobs); free(tids); return ORACLE_ENOMEM; }
    for (int t = 1; t < nt; ++t) ok[t] = (pthread_create(&tids[t], NULL, worker, &jobs[t]) == 0);
    if (nt > 0) worker(&jobs[0]);
    for (int t = 1; t < nt; ++t) {
        if (ok[t]) pthread_join(tids[t], NULL);
        else worker(&jobs[t]);
    }
    free(ok);

    if (row1 == m && (m & 63)) out[(m - 1) >> 6] &= (((uint64_t)1) << (m & 63)) - 1;
    free(jobs);
    free(tids);
    free(xr);
    return ORACLE_OK;
}

/* All m rows. out must hold ceil(m/64) words; it is fully written. */
int pa_oracle_hash(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key, uint64_t *out, int threads) {
    if (!out || m == 0) return ORACLE_EINVAL;
    memset(out, 0, (size_t)nwords(m) * sizeof(uint64_t));
    return pa_oracle_hash_rows(n, m, seed, key, 0, m, out, threads);
}

/* One output bit, for spot checks at sizes where all rows would take too long. */
int pa_oracle_row(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key, uint64_t i) {
    if (n == 0 || m == 0 || i >= m || !seed || !key) return ORACLE_EINVAL;
    uint64_t nw = nwords(n);
    uint64_t *xr = (uint64_t *)calloc(nw, sizeof(uint64_t));
    if (!xr) return ORACLE_ENOMEM;
    for (uint64_t j = 0; j < n; ++j)
        if (get_bit(key, n - 1 - j)) xr[j >> 6] |= ((uint64_t)1) << (j & 63);
    int b = row_parity(n, m, seed, xr, i);
    free(xr);
    return b;
}

/*
 * Several rows at once (sorted or not): rows[k] -> bits[k] in {0,1}. The
 * reversed key is built once, rows are split across threads.
 */
typedef struct {
    uint64_t n, m;
    const uint64_t *seed, *xr, *rows;
    uint8_t *bits;
    uint64_t k0, k1;
} rows_job_t;

static void *rows_worker(void *arg) {
    rows_job_t *jb = (rows_job_t *)arg;
    for (uint64_t k = jb->k0; k < jb->k1; ++k)
        jb->bits[k] = (uint8_t)row_parity(jb->n, jb->m, jb->seed, jb->xr, jb->rows[k]);
    return NULL;
}

int pa_oracle_rows(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key, const uint64_t *rows,
                   uint64_t nrows, uint8_t *bits, int threads) {
    if (n == 0 || m == 0 || !seed || !key || (nrows && (!rows || !bits))) return ORACLE_EINVAL;
    for (uint64_t k = 0; k < nrows; ++k)
        if (rows[k] >= m) return ORACLE_EINVAL;
    uint64_t nw = nwords(n);
    uint64_t *xr = (uint64_t *)calloc(nw, sizeof(uint64_t));
    if (!xr) return ORACLE_ENOMEM;
    for (uint64_t j = 0; j < n; ++j)
        if (get_bit(key, n - 1 - j)) xr[j >> 6] |= ((uint64_t)1) << (j & 63);
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > nrows) threads = nrows ? (int)nrows : 1;
    rows_job_t *jobs = (rows_job_t *)calloc((size_t)threads, sizeof(rows_job_t));
    pthread_t *tids = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) { free(xr); free(jobs); free(tids); return ORACLE_ENOMEM; }
    uint64_t per = (nrows + (uint64_t)threads - 1) / (uint64_t)threads;
    for (int t = 0; t < threads; ++t) {
        uint64_t a = (uint64_t)t * per, b = a + per;
        if (a > nrows) a = nrows;
        if (b > nrows) b = nrows;
        jobs[t] = (rows_job_t){n, m, seed, xr, rows, bits, a, b};
    }
    int *ok = (int *)calloc((size_t)threads, sizeof(int));
    for (int t = 1; t < threads; ++t) ok[t] = (pthread_create(&tids[t], NULL, rows_worker, &jobs[t]) == 0);
    rows_worker(&jobs[0]);
    for (int t = 1; t < threads; ++t) {
        if (ok[t]) pthread_join(tids[t], NULL);
        else rows_worker(&jobs[t]);
    }
    free(ok);
    free(jobs);
    free(tids);
    free(xr);
    return ORACLE_OK;
}

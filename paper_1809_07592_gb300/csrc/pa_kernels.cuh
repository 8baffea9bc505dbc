// pa_kernels.cuh -- the pass kernels of the FFT Toeplitz hash.
//
// Index conventions for a transform of complex length L = L1 * L2 (two
// levels) or L1 * L2 * L3 (three levels). Element t of a length-L vector lives
// at offset t of its work slot; a pass at level j with transform length LEN and
// stride S treats the slot as blocks of LEN*S elements, each holding S
// interleaved columns of LEN elements (element a of column u at a*S + u).
//
//   forward level j (decimation in frequency, paper Algorithm 1's "row FFT
//   then twiddle W[i*j]"): X[k] = sum_a x[a] w_LEN^{a k}, then
//   X[k] *= w_{LEN*S}^{k u}, stored back at k*S + u.
//   inverse level j: x[k] *= w_{LEN*S}^{-k u}, then the unscaled inverse DFT.
//
// The innermost level (S = 1, contiguous) fuses the last forward step, the
// pointwise product with the cached seed spectrum (Eq. 4's FFT(V) . FFT(X))
// and the first inverse step. The seed spectrum already carries the 1/L of
// the inverse transform.
//
// Encoding (the value that is rounded): key bits x_j in {0,1}; seed bits
// enter as sigma = 1 - 2 s in {+1,-1} and are rotated so the wanted window of
// the linear convolution lands at positions 0..m-1:
//     r_i = sum_j sigma[i - j + n - 1] x_j = P - 2 c_i,
// where c_i = sum_j s[i-j+n-1] x_j is the GF(2) row count and P = popcount(x).
// So y_i = c_i mod 2 = rint((P - r_i)/2) mod 2, and since 4 | (P - P mod 4)
// only P mod 4 enters: y_i = rint(w_i) mod 2 with w_i = ((P mod 4) - r_i)/2.
// |r_i| grows like sqrt(n) instead of n, which keeps FP32 rounding far from
// the 0.5 cliff (the precision concern of the paper's Section 5).
#pragma once

#include "bulk.cuh"
#include "fft_core.cuh"

namespace pa {

// Resident CTAs requested per SM for a CTA of `threads` threads: enough for 1024
// threads, so the register allocation stays <= 64 per thread and at least two
// CTAs overlap their load, transform and store phases.
__host__ __device__ constexpr int min_blocks(int threads) { return threads >= 1024 ? 1 : (1024 / threads > 16 ? 16 : 1024 / threads); }
// The fused innermost passes ask for 512 resident threads per SM (<= 128
// registers each; at most 16 CTAs). In single precision (8-byte elements) they ask for 768, at
// most 8 CTAs: measured on the DV-QKD lengths, 17-31 % faster than 512 (more CTAs
// overlap their barrier and load phases) with no spills. Rows of 5120 values
// (CTAs of 320 threads) ask for three CTAs (960 threads, at most 68 registers)
// and rows of 4608 (288 threads) for four (1152 threads, at most 56), both without
// spills: the pass ran 8.8 % faster on the DV-QKD batches with three CTAs than with
// two, and 0.6 % faster again with the fourth for 4608; four CTAs of 320 threads
// and three of 384 (6144 values) spill and were slower. The two-row split kernel
// keeps 512 (it spills above).
__host__ __device__ constexpr int min_blocks_inner(int threads, int elem_bytes = 16) {
    return elem_bytes > 8 ? (threads >= 512 ? 1 : (512 / threads > 16 ? 16 : 512 / threads))
                          : (threads >= 768 ? 1
                                            : threads == 288 ? 4
                                            : threads == 320 ? 3
                                                             : (768 / threads > 8 ? 8 : 768 / threads));
}

// Rounding to the nearest integer (ties to even) by adding and subtracting
// 1.5 * 2^(mantissa bits): exact for |x| < 2^22 (float) / 2^51 (double); the
// integer's parity is the lowest bit of the sum's encoding.
template <typename T> struct Magic;
template <> struct Magic<float> { static constexpr float v = 12582912.0f, limit = 2097152.0f; };
template <> struct Magic<double> { static constexpr double v = 6755399441055744.0, limit = 1125899906842624.0; };
__device__ __forceinline__ uint32_t low_bit(float x) { return __float_as_uint(x) & 1u; }
__device__ __forceinline__ uint32_t low_bit(double x) { return (uint32_t)__double_as_longlong(x) & 1u; }

// Encoding of inputs and decoding of outputs per arithmetic.
// Complex: key bits 0/1 in the real (key 2p) and imaginary (key 2p+1) parts,
// seed as +-1; the decoded value is w = ((P mod 4) - r)/2 (see above).
// Zp: key 2p + 2^32 * key 2p+1 packed in one residue, seed as 0/1; the
// convolution counts c_a, c_b < 2^32 come out exactly as the low and high
// halves of the canonical residue.
template <typename T> struct Enc {
    using E = cx<T>;
    using M = T;  // margin accumulator
    static __device__ __forceinline__ E key_pair(uint32_t ba, uint32_t bb) {
        return Arith<T>::mk(ba ? (T)1 : (T)0, bb ? (T)1 : (T)0);
    }
    static __device__ __forceinline__ E seed(bool in_range, uint32_t bit) {
        return Arith<T>::mk(in_range ? (bit ? (T)-1 : (T)1) : (T)0, (T)0);
    }
    static __device__ __forceinline__ E seed_pair(bool in0, uint32_t b0, bool in1, uint32_t b1) {
        return Arith<T>::mk(in0 ? (b0 ? (T)-1 : (T)1) : (T)0, in1 ? (b1 ? (T)-1 : (T)1) : (T)0);
    }
    // bits and margins of the two values carried by v (valid_b: the imaginary part's own range)
    static __device__ __forceinline__ void decode(E v, uint32_t popa, uint32_t popb, bool valid, bool &bit_a,
                                                  bool &bit_b, M &ma, M &mb) {
        decode2(v, popa, popb, valid, valid, bit_a, bit_b, ma, mb);
    }
    static __device__ __forceinline__ void decode2(E v, uint32_t popa, uint32_t popb, bool valid_a, bool valid_b,
                                                   bool &bit_a, bool &bit_b, M &ma, M &mb) {
        const T wa = ((T)(popa & 3u) - v.x) * (T)0.5, wb = ((T)(popb & 3u) - v.y) * (T)0.5;
        const T fa = wa + Magic<T>::v, fb = wb + Magic<T>::v;  // rint via the 1.5*2^p addition
        bit_a = valid_a && low_bit(fa);
        bit_b = valid_b && low_bit(fb);
        // beyond the limit the parity is not resolvable: report a margin of 1 so the guard escalates
        if (valid_a) ma = fmax(ma, fabs(wa) < Magic<T>::limit ? fabs(wa - (fa - Magic<T>::v)) : (T)1);
        if (valid_b) mb = fmax(mb, fabs(wb) < Magic<T>::limit ? fabs(wb - (fb - Magic<T>::v)) : (T)1);
    }
};
template <> struct Enc<Zp> {
    using E = cx<Zp>;
    using M = float;
    static __device__ __forceinline__ E key_pair(uint32_t ba, uint32_t bb) { return (E)ba | ((E)bb << 32); }
    static __device__ __forceinline__ E seed(bool in_range, uint32_t bit) { return (in_range && bit) ? 1ull : 0ull; }
    // (the exact transform has no half-length packing of one key: its values are not complex)
    static __device__ __forceinline__ E seed_pair(bool, uint32_t, bool, uint32_t) { return 0ull; }
    static __device__ __forceinline__ void decode(E v, uint32_t, uint32_t, bool valid, bool &bit_a, bool &bit_b, M &,
                                                  M &) {
        bit_a = valid && (v & 1ull);
        bit_b = valid && ((v >> 32) & 1ull);
    }
    static __device__ __forceinline__ void decode2(E v, uint32_t, uint32_t, bool valid_a, bool valid_b, bool &bit_a,
                                                   bool &bit_b, M &, M &) {
        bit_a = valid_a && (v & 1ull);
        bit_b = valid_b && ((v >> 32) & 1ull);
    }
};

// ---------------------------------------------------------------------------
// Bit staging for the level-1 forward passes: per row, the CTA's COLS input bits
// (low 16 bits: key or key a; high 16 bits: key b or seed) after the transform's
// shared memory.
template <typename T, int LEN, int COLS>
__device__ __forceinline__ uint32_t *key_stage(unsigned char *smem_raw) {
    return reinterpret_cast<uint32_t *>(smem_raw + smem_elems<LEN, COLS>() * sizeof(cx<T>));
}
template <typename T, int LEN, int COLS>
constexpr size_t stage_bytes() { return (size_t)LEN * sizeof(uint32_t); }

// Two per-thread counters reduced over the CTA (sum, or max when MAX): warp reductions,
// then warp 0 over the warps' partial results (kept in scratch, 64 words of shared
// memory). The totals are valid in thread 0. Every thread of the CTA must call it (it
// holds a barrier). The per-key counters of a batch (key popcounts, rounding margins)
// are accumulated with one atomic per key and CTA this way: one atomic per warp on the
// same few words from thousands of CTAs at once queues up in the memory system and
// measurably slows the whole pass.
template <bool MAX>
__device__ __forceinline__ void cta_reduce2(uint32_t &a, uint32_t &b, uint32_t *scratch) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = MAX ? __reduce_max_sync(0xffffffffu, a) : __reduce_add_sync(0xffffffffu, a);
    b = MAX ? __reduce_max_sync(0xffffffffu, b) : __reduce_add_sync(0xffffffffu, b);
    if (lane == 0) {
        scratch[warp] = a;
        scratch[32 + warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        const uint32_t nw = blockDim.x >> 5;
        a = lane < nw ? scratch[lane] : 0u;
        b = lane < nw ? scratch[32 + lane] : 0u;
        a = MAX ? __reduce_max_sync(0xffffffffu, a) : __reduce_add_sync(0xffffffffu, a);
        b = MAX ? __reduce_max_sync(0xffffffffu, b) : __reduce_add_sync(0xffffffffu, b);
    }
}

// Single keys in half-length transforms: transform element t carries key bits 2t
// (real part) and 2t+1 (imaginary part). even_bits gathers the even-position bits of
// x into the low 16 bits; spread_bits is its inverse (low 16 bits to even positions).
__device__ __forceinline__ uint32_t even_bits(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    return (x | (x >> 8)) & 0x0000FFFFu;
}
__device__ __forceinline__ uint32_t spread_bits(uint32_t x) {
    x &= 0x0000FFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    return (x | (x << 1)) & 0x55555555u;
}

// COLS bits of v starting at bit t0 (t0 % COLS == 0, so they sit in one word);
// bits at or past nbits read as 0.
template <int COLS>
__device__ __forceinline__ uint32_t aligned_bits(const uint64_t *v, uint64_t nbits, uint64_t t0) {
    if (t0 >= nbits) return 0u;
    uint32_t w = (uint32_t)(__ldg(v + (t0 >> 6)) >> (t0 & 63)) & ((1u << COLS) - 1u);
    const uint64_t left = nbits - t0;
    if (left < COLS) w &= (1u << left) - 1u;
    return w;
}

// cnt <= 32 bits of v starting at an arbitrary bit position pos; bits at or past nbits read as 0.
__device__ __forceinline__ uint32_t bits_at(const uint64_t *v, uint64_t nbits, uint64_t pos, uint32_t cnt) {
    if (pos >= nbits || cnt == 0) return 0u;
    const uint64_t q = pos >> 6;
    const uint32_t r = (uint32_t)(pos & 63);
    uint64_t x = __ldg(v + q) >> r;
    if (r + cnt > 64 && ((q + 1) << 6) < nbits) x |= __ldg(v + q + 1) << (64 - r);
    uint32_t w = (uint32_t)x & (cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u));
    const uint64_t left = nbits - pos;
    if (left < cnt) w &= (1u << left) - 1u;
    return w;
}

// ---------------------------------------------------------------------------
// Level-1 forward pass from packed key bits. Grid (S/COLS, pairs); pair p
// carries key 2p in the real part and key 2p+1 (if any) in the imaginary part.
// PACK: slot p carries one key, p, in a half-length transform: element t is key
// bits 2t (real part) and 2t+1 (imaginary part).
template <typename T, int LEN, int COLS, int E, bool PACK = false>
__global__ void __launch_bounds__(COLS * LEN / E, min_blocks(COLS * LEN / E))
    k_fwd_keys(const uint64_t *__restrict__ keys, uint32_t nkeys, uint64_t kstride, uint64_t n,
               cx<T> *__restrict__ W, uint64_t L, TwTab<T> tw, uint32_t *__restrict__ popc, uint64_t koff) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    const uint32_t col = threadIdx.x % COLS, tq = threadIdx.x / COLS;
    const uint64_t S = L >> ilog2(LEN);
    const uint64_t u = (uint64_t)blockIdx.x * COLS + col;
    const uint32_t pair = blockIdx.y;
    const bool has_b = 2 * pair + 1 < nkeys;
    // Stage the CTA's COLS bits of every row of both keys in shared memory first:
    // one word load per row instead of one per element, all in flight together.
    uint32_t *stage = key_stage<T, LEN, COLS>(smem_raw);
    const uint64_t u0 = (uint64_t)blockIdx.x * COLS;
    uint32_t ca = 0, cb = 0;  // the CTA's share of each key's popcount P (the CTAs tile every bit once)
    // The transform's input element t is key bit koff + t (koff = 0, or m for the modified
    // Toeplitz hash, whose Toeplitz block multiplies key bits m .. n-1).
    const uint64_t nk = n + koff;
    const bool aligned = (koff % COLS) == 0;
    const uint64_t *xa = keys + (uint64_t)(PACK ? pair : 2 * pair) * kstride, *xb = xa + kstride;
    for (uint32_t a = threadIdx.x; a < LEN; a += blockDim.x) {
        const uint64_t t0 = (uint64_t)a * S + u0 + koff;  // S % 64 == 0: aligned COLS bits sit in one word
        uint32_t wa, wb = 0u;
        if constexpr (PACK) {  // 2*COLS key bits from 2*(a*S + u0): the even ones real, the odd ones imaginary
            const uint32_t c = bits_at(xa, nk, 2 * ((uint64_t)a * S + u0) + koff, 2 * COLS);
            wa = even_bits(c);
            wb = even_bits(c >> 1);
        } else if (aligned) {
            wa = aligned_bits<COLS>(xa, nk, t0);
            if (has_b) wb = aligned_bits<COLS>(xb, nk, t0);
        } else {
            wa = bits_at(xa, nk, t0, COLS);
            if (has_b) wb = bits_at(xb, nk, t0, COLS);
        }
        stage[a] = wa | (wb << 16);
        ca += __popc(wa);
        cb += __popc(wb);
    }
    __shared__ uint32_t red[64];
    cta_reduce2<false>(ca, cb, red);  // also publishes the staged rows
    if (threadIdx.x == 0 && (ca | cb)) {
        if (PACK) {
            atomicAdd(popc + pair, ca + cb);
        } else {
            if (ca) atomicAdd(popc + 2 * pair, ca);
            if (cb) atomicAdd(popc + 2 * pair + 1, cb);
        }
    }
    cx<T> v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const uint32_t w2 = stage[idx_r0<LEN, E>(tq, s)];
        v[s] = Enc<T>::key_pair((w2 >> col) & 1u, (w2 >> (16 + col)) & 1u);
    }
    cta_fft<T, LEN, COLS, E, false>(sm, v, tq, col, tw);
    cx<T> *w = W + (uint64_t)pair * L;
    // k = tq + s*TC: w_L^{k u} = w_L^{tq u} * (w_L^{TC u})^s
    twiddle_chain<T, false, E>(v, tw, (uint32_t)(tq * u), (uint32_t)((LEN / E) * u));
#pragma unroll
    for (int s = 0; s < E; ++s) w[(uint64_t)idx_e<LEN, E>(tq, s) * S + u] = v[s];
}

// Level-1 forward pass of the rotated, +-1 encoded seed (real input). PACK: the
// seed of a length-2L convolution in a length-L transform, element t carrying
// rotated positions 2t (real part) and 2t+1 (imaginary part).
template <typename T, int LEN, int COLS, int E, bool PACK = false>
__global__ void __launch_bounds__(COLS * LEN / E, min_blocks(COLS * LEN / E))
    k_fwd_seed(const uint64_t *__restrict__ seed, uint64_t n, uint64_t m, cx<T> *__restrict__ W, uint64_t L,
               TwTab<T> tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    const uint32_t col = threadIdx.x % COLS, tq = threadIdx.x / COLS;
    const uint64_t S = L >> ilog2(LEN);
    const uint64_t u = (uint64_t)blockIdx.x * COLS + col;
    const uint64_t sbits = n + m - 1;
    cx<T> v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const uint64_t pos = (uint64_t)idx_r0<LEN, E>(tq, s) * S + u;
        if constexpr (PACK) {
            const uint64_t L2 = 2 * L;
            uint32_t bit[2];
            bool in_range[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint64_t j = 2 * pos + h + n - 1;  // seed index at rotated position 2*pos + h
                if (j >= L2) j -= L2;
                in_range[h] = j < sbits;
                bit[h] = in_range[h] ? (uint32_t)(__ldg(seed + (j >> 6)) >> (j & 63)) & 1u : 0u;
            }
            v[s] = Enc<T>::seed_pair(in_range[0], bit[0], in_range[1], bit[1]);
        } else {
            uint64_t j = pos + n - 1;  // seed index whose value sits at rotated position pos
            if (j >= L) j -= L;
            const bool in_range = j < sbits;
            const uint32_t bit = in_range ? (uint32_t)(__ldg(seed + (j >> 6)) >> (j & 63)) & 1u : 0u;
            v[s] = Enc<T>::seed(in_range, bit);
        }
    }
    cta_fft<T, LEN, COLS, E, false>(sm, v, tq, col, tw);
    twiddle_chain<T, false, E>(v, tw, (uint32_t)(tq * u), (uint32_t)((LEN / E) * u));
#pragma unroll
    for (int s = 0; s < E; ++s) W[(uint64_t)idx_e<LEN, E>(tq, s) * S + u] = v[s];
}

// Middle-level strided pass (three-level plans only), forward or inverse.
// S is the innermost length (the stride of this pass); blocks of LEN*S elements;
// w_{LEN*S}^e = w_L^{e * mult} with mult = L / (LEN*S). Grid (S/COLS, blocks * pairs).
template <typename T, int LEN, int COLS, int E, bool INV>
__global__ void __launch_bounds__(COLS * LEN / E, min_blocks(COLS * LEN / E))
    k_mid(cx<T> *__restrict__ W, uint64_t L, uint32_t S, uint32_t mult, TwTab<T> tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    const uint32_t col = threadIdx.x % COLS, tq = threadIdx.x / COLS;
    const uint64_t blk_len = (uint64_t)LEN * S;
    const uint64_t nblk = L / blk_len;
    const uint64_t pair = blockIdx.y / nblk, blk = blockIdx.y % nblk;
    const uint32_t u = blockIdx.x * COLS + col;
    cx<T> *w = W + pair * L + blk * blk_len;
    cx<T> v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const uint32_t a = INV ? idx_e<LEN, E>(tq, s) : idx_r0<LEN, E>(tq, s);
        v[s] = w[(uint64_t)a * S + u];
    }
    if (INV) twiddle_chain<T, true, E>(v, tw, (tq * u) * mult, ((LEN / E) * u) * mult);
    cta_fft<T, LEN, COLS, E, INV>(sm, v, tq, col, tw);
    if (!INV) twiddle_chain<T, false, E>(v, tw, (tq * u) * mult, ((LEN / E) * u) * mult);
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const uint32_t a = INV ? idx_r0<LEN, E>(tq, s) : idx_e<LEN, E>(tq, s);
        w[(uint64_t)a * S + u] = v[s];
    }
}

// Innermost level: contiguous rows of LEN elements. MODE 0: forward, times
// the seed spectrum, inverse (the fused convolution step). MODE 1: forward
// only, scaled by 1/L, written as the seed spectrum.
template <typename T, int LEN, int E, int MODE>
__global__ void __launch_bounds__(LEN / E, min_blocks_inner(LEN / E, sizeof(cx<T>)))
    k_middle(cx<T> *__restrict__ W, cx<T> *__restrict__ spec, uint64_t L, TwTab<T> tw, cx<T> scale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    const uint32_t tq = threadIdx.x;
    const uint64_t row = blockIdx.x, pair = blockIdx.y;
    // thread tq's elements sit at compile-time offsets from element tq of the row
    cx<T> *wt = W + pair * L + row * LEN + tq;
    cx<T> *spt = spec + row * LEN + tq;
    cx<T> v[E];
    if constexpr (Plan<LEN, E>::RO == 1) {
#pragma unroll
        for (int s = 0; s < E; ++s) v[s] = wt[idx_r0<LEN, E>(0, s)];
        cta_fft<T, LEN, 1, E, false>(sm, v, tq, 0, tw);
    } else {
        cta_fft_fwd_odd<T, LEN, E>(sm, v, tq, tw, [&](uint32_t o) { return wt[o]; });
    }
    if constexpr (MODE == 1) {
#pragma unroll
        for (int s = 0; s < E; ++s) spt[idx_e<LEN, E>(0, s)] = Arith<T>::mul(v[s], scale);
    } else {
#pragma unroll
        for (int s = 0; s < E; ++s) v[s] = Arith<T>::mul(v[s], spt[idx_e<LEN, E>(0, s)]);
        __syncthreads();  // the forward transform's last shared-memory reads are done
        if constexpr (Plan<LEN, E>::RO == 1) {
            cta_fft<T, LEN, 1, E, true>(sm, v, tq, 0, tw);
#pragma unroll
            for (int s = 0; s < E; ++s) wt[idx_r0<LEN, E>(0, s)] = v[s];
        } else {
            cta_fft_inv_odd<T, LEN, E>(sm, v, tq, tw, [&](uint32_t o, cx<T> x) { wt[o] = x; });
        }
    }
}

// Word type for COLS output bits.
template <int COLS> struct BitsWord;
template <> struct BitsWord<8> { using type = uint8_t; };
template <> struct BitsWord<16> { using type = uint16_t; };
template <> struct BitsWord<32> { using type = uint32_t; };

__device__ __forceinline__ float margin_to_float(float x) { return x; }
__device__ __forceinline__ float margin_to_float(double x) { return __double2float_ru(x); }

// Round, mod 2 and pack the outputs of the level-1 inverse transform of one column
// (pair form): v holds rows t1 = idx_r0(tq, s) of column u = u0 + col, the real part
// belonging to key ka with ma_bits outputs, the imaginary part to key kb (if has_b) with
// mb_bits outputs (the uneven batch pairs blocks of different lengths; a plan's pairs
// have ma_bits = mb_bits = m). Output bit i = t1*S + u of a key is element i of the
// convolution window; bits past the key's outputs are written 0. Each key's rounding
// margin max |w - rint(w)| over its outputs goes to margin_bits[ka] / [kb] (float bits,
// atomicMax; margins are >= 0, so integer order is float order). With xkeys, the bits
// are XORed with key bits 0 .. m-1 (the identity block of the modified hash, Eq. 3).
template <typename T, int LEN, int COLS, int E>
__device__ __forceinline__ void pack_pair_bits(const cx<T> *v, uint32_t tq, uint32_t col, uint64_t S, uint64_t u0,
                                               uint64_t ma_bits, uint64_t mb_bits, uint32_t popa, uint32_t popb,
                                               uint32_t ka, uint32_t kb, bool has_b,
                                               typename BitsWord<COLS>::type *oa,
                                               typename BitsWord<COLS>::type *ob, uint32_t *margin_bits,
                                               const uint64_t *xkeys, uint64_t xstride) {
    using word_t = typename BitsWord<COLS>::type;
    const uint32_t lane = threadIdx.x & 31;
    // 32-bit positions (t1*S + u < L <= 2^28). Rows at or past the end of the last output word
    // are not decoded; the test uses the warp's first row of each slot (rows grow with tq, so
    // the whole warp is past the end when its first row is), which keeps it warp-uniform: the
    // ballots below need every lane. The bound is taken once as a row count, and where a
    // thread's rows grow with the slot (one radix-E last stage) the loop stops at the first
    // slot past it.
    const uint32_t S32 = (uint32_t)S, u032 = (uint32_t)u0;
    const uint32_t ma32 = (uint32_t)ma_bits, mb32 = has_b ? (uint32_t)mb_bits : 0u;
    const uint32_t mwa = (uint32_t)(((ma_bits + 63) >> 6) << 6), mwb = has_b ? (uint32_t)(((mb_bits + 63) >> 6) << 6) : 0u;
    const uint32_t mw = mwa > mwb ? mwa : mwb;
    const uint32_t tq0 = (threadIdx.x & ~31u) / COLS;  // the warp's first tq
    const uint32_t nrow = mw > u032 ? (mw - u032 + S32 - 1u) / S32 : 0u;  // rows t1 with t1*S + u0 < mw
    typename Enc<T>::M ma = 0, mb = 0;
    [[maybe_unused]] float wa_max = 0.f, wb_max = 0.f;  // single precision: largest |w| of each key
    [[maybe_unused]] const float2 half_p = make_float2(0.5f * (float)(popa & 3u), 0.5f * (float)(popb & 3u));
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const uint32_t t1 = idx_r0<LEN, E>(tq, s);
        if constexpr (Plan<LEN, E>::r0 == E) {  // t1 = tq + s*TC: every later slot is past the bound too
            if (idx_r0<LEN, E>(tq0, s) >= nrow) break;
        } else {
            if (idx_r0<LEN, E>(tq0, s) >= nrow) continue;
        }
        const uint32_t row0 = t1 * S32 + u032;  // output bit of this row's first column
        const bool valid_a = row0 + col < ma32, valid_b = row0 + col < mb32;
        bool bit_a, bit_b;
        if constexpr (std::is_same<T, float>::value) {
            // w = ((P mod 4) - r)/2 for both keys at once; rint by the 1.5*2^23 addition (exact for |w| < 2^22)
            const float2 w = f2_fma(v[s], make_float2(-0.5f, -0.5f), half_p);
            const float2 f = f2_add(w, make_float2(Magic<float>::v, Magic<float>::v));
            const float2 d = f2_sub(w, f2_sub(f, make_float2(Magic<float>::v, Magic<float>::v)));
            bit_a = valid_a && (__float_as_uint(f.x) & 1u);
            bit_b = valid_b && (__float_as_uint(f.y) & 1u);
            ma = fmaxf(ma, valid_a ? fabsf(d.x) : 0.f);
            mb = fmaxf(mb, valid_b ? fabsf(d.y) : 0.f);
            wa_max = fmaxf(wa_max, valid_a ? fabsf(w.x) : 0.f);
            wb_max = fmaxf(wb_max, valid_b ? fabsf(w.y) : 0.f);
        } else {
            Enc<T>::decode2(v[s], popa, popb, valid_a, valid_b, bit_a, bit_b, ma, mb);
        }
        const uint32_t ba = __ballot_sync(0xffffffffu, bit_a);
        const uint32_t bb = __ballot_sync(0xffffffffu, bit_b);
        if (col == 0) {
            const uint32_t ci = row0 / COLS;  // output chunk of this row's COLS bits
            const uint32_t msk = (COLS == 32) ? 0xffffffffu : ((1u << COLS) - 1u);
            uint32_t ya = (ba >> lane) & msk, yb = (bb >> lane) & msk;  // lane = group * COLS
            if (xkeys) {  // modified Toeplitz hash (Eq. 3): the identity block adds key bits 0 .. m-1
                ya ^= aligned_bits<COLS>(xkeys + (uint64_t)ka * xstride, ma_bits, row0);
                if (has_b) yb ^= aligned_bits<COLS>(xkeys + (uint64_t)kb * xstride, mb_bits, row0);
            }
            if (row0 < mwa) oa[ci] = (word_t)ya;
            if (row0 < mwb) ob[ci] = (word_t)yb;
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        // beyond the exact range of the rounding the parity is not resolvable: a margin of 1 escalates
        if (wa_max >= Magic<float>::limit) ma = 1.f;
        if (wb_max >= Magic<float>::limit) mb = 1.f;
    }
    uint32_t fa = __float_as_uint(margin_to_float(ma)), fb = __float_as_uint(margin_to_float(mb));
    __shared__ uint32_t red[64];
    cta_reduce2<true>(fa, fb, red);
    if (threadIdx.x == 0) {
        atomicMax(margin_bits + ka, fa);
        if (has_b) atomicMax(margin_bits + kb, fb);
    }
}

// Level-1 inverse pass with the post-processing step of the paper's Fig. 2 (the
// inverse transform's output rounded to integers, then reduced mod 2): round, mod 2, pack.
// Output bit i = element i of the convolution window; bits >= m are written 0.
// Each key's rounding margin max |w - rint(w)| goes to margin_bits (float bits,
// atomicMax; all margins are >= 0 so integer order equals float order).
// PACK: slot p holds one key p of a half-length transform; element t carries output
// bits 2t (real part) and 2t+1 (imaginary part).
template <typename T, int LEN, int COLS, int E, bool PACK = false>
__global__ void __launch_bounds__(COLS * LEN / E, min_blocks(COLS * LEN / E))
    k_inv_bits(const cx<T> *__restrict__ W, uint64_t L, uint64_t m, uint32_t nkeys,
               const uint32_t *__restrict__ popc, uint32_t *__restrict__ margin_bits, uint64_t *__restrict__ out,
               uint64_t ostride, TwTab<T> tw, const uint64_t *__restrict__ xkeys, uint64_t xstride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    using word_t = typename BitsWord<COLS>::type;
    const uint32_t col = threadIdx.x % COLS, tq = threadIdx.x / COLS;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t S = L >> ilog2(LEN);
    const uint64_t u0 = (uint64_t)blockIdx.x * COLS;
    const uint64_t u = u0 + col;
    const uint32_t pair = blockIdx.y;
    const uint32_t ka = PACK ? pair : 2 * pair, kb = 2 * pair + 1;
    const bool has_b = !PACK && kb < nkeys;
    const cx<T> *w = W + (uint64_t)pair * L;
    cx<T> v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = w[(uint64_t)idx_e<LEN, E>(tq, s) * S + u];
    twiddle_chain<T, true, E>(v, tw, (uint32_t)(tq * u), (uint32_t)((LEN / E) * u));
    cta_fft<T, LEN, COLS, E, true>(sm, v, tq, col, tw);

    const uint32_t popa = popc[ka];
    const uint32_t popb = PACK ? popa : (has_b ? popc[kb] : 0u);
    word_t *oa = reinterpret_cast<word_t *>(out + (uint64_t)ka * ostride);
    word_t *ob = reinterpret_cast<word_t *>(out + (uint64_t)kb * ostride);
    if constexpr (PACK) {
        typename Enc<T>::M ma = 0, mb = 0;
        [[maybe_unused]] float w_max = 0.f;
        [[maybe_unused]] const float half_p = 0.5f * (float)(popa & 3u);
        // chunk ci: the row's COLS elements t = t1*S + u0 + c, i.e. output bits 2*(t1*S + u0) .. +2*COLS;
        // 32-bit positions, and the warp-uniform skip of rows past the last output word as in pack_pair_bits
        using word2_t = typename BitsWord<2 * COLS>::type;
        word2_t *o2 = reinterpret_cast<word2_t *>(out + (uint64_t)ka * ostride);
        const uint32_t S32 = (uint32_t)S, u032 = (uint32_t)u0, m32 = (uint32_t)m;
        const uint32_t mw = (uint32_t)(((m + 63) >> 6) << 6);  // output bits up to the end of the last word
        const uint32_t tq0 = (threadIdx.x & ~31u) / COLS;
        const uint32_t half = mw >> 1;  // rows t1 with 2*(t1*S + u0) < mw: t1 < nrow
        const uint32_t nrow = half > u032 ? (half - u032 + S32 - 1u) / S32 : 0u;
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const uint32_t t1 = idx_r0<LEN, E>(tq, s);
            if constexpr (Plan<LEN, E>::r0 == E) {
                if (idx_r0<LEN, E>(tq0, s) >= nrow) break;
            } else {
                if (idx_r0<LEN, E>(tq0, s) >= nrow) continue;
            }
            const uint32_t row0 = t1 * S32 + u032;
            const uint32_t t = row0 + col;
            const bool ve = 2 * t < m32, vo = 2 * t + 1 < m32;
            bool bit_e, bit_o;
            if constexpr (std::is_same<T, float>::value) {
                const float2 w = f2_fma(v[s], make_float2(-0.5f, -0.5f), make_float2(half_p, half_p));
                const float2 f = f2_add(w, make_float2(Magic<float>::v, Magic<float>::v));
                const float2 d = f2_sub(w, f2_sub(f, make_float2(Magic<float>::v, Magic<float>::v)));
                bit_e = ve && (__float_as_uint(f.x) & 1u);
                bit_o = vo && (__float_as_uint(f.y) & 1u);
                ma = fmaxf(ma, ve ? fabsf(d.x) : 0.f);
                mb = fmaxf(mb, vo ? fabsf(d.y) : 0.f);
                w_max = fmaxf(w_max, fmaxf(ve ? fabsf(w.x) : 0.f, vo ? fabsf(w.y) : 0.f));
            } else {
                Enc<T>::decode2(v[s], popa, popa, ve, vo, bit_e, bit_o, ma, mb);
            }
            const uint32_t be = __ballot_sync(0xffffffffu, bit_e);
            const uint32_t bo = __ballot_sync(0xffffffffu, bit_o);
            if (col == 0 && 2 * row0 < mw) {
                const uint32_t ci = row0 / COLS;
                const uint32_t msk = (1u << COLS) - 1u;
                uint32_t y = spread_bits((be >> lane) & msk) | (spread_bits((bo >> lane) & msk) << 1);
                if (xkeys) y ^= bits_at(xkeys + (uint64_t)ka * xstride, m, 2 * (uint64_t)row0, 2 * COLS);
                o2[ci] = (word2_t)y;
            }
        }
        if constexpr (std::is_same<T, float>::value) {
            if (w_max >= Magic<float>::limit) ma = 1.f;  // parity not resolvable: escalate
        }
        uint32_t f = __float_as_uint(margin_to_float(ma > mb ? ma : mb)), unused = 0u;
        __shared__ uint32_t red[64];
        cta_reduce2<true>(f, unused, red);
        if (threadIdx.x == 0) atomicMax(margin_bits + ka, f);
        return;
    }
    pack_pair_bits<T, LEN, COLS, E>(v, tq, col, S, u0, m, m, popa, popb, ka, kb, has_b, oa, ob, margin_bits, xkeys,
                                    xstride);
}

// The level-1 inverse pass of key pairs (FP32, pair form) as a persistent kernel whose
// input tiles are staged by the TMA: tile t is the COLS x LEN block of columns
// u0 .. u0+COLS-1 of pair t / (S / COLS), copied by one tiled copy into shared memory.
// The copy of a CTA's next tile is issued as soon as every thread has read the current
// one, so a copy is in flight while the tile is transformed and decoded: the pass keeps
// enough bytes in flight without spending registers on them. The arithmetic is
// k_inv_bits's, step for step. The tensor map describes the work buffer as a
// (pairs * LEN) x S array of 8-byte elements (row a of pair p at row p*LEN + a).
//
// Tiles are handed out by a ticket counter (ctl[1]), so a CTA that starts late, behind
// another stream's kernel, just takes fewer tiles. Every CTA counts itself out on ctl[2]
// when it leaves; the last one resets both counters for the next launch (launches that
// share ctl run in stream order). A copy wait that runs out of time sets bit 0 of ctl[0]
// and the CTA leaves after a second bounded wait for that copy. expire_ns != 0 is a test
// hook for that path: no CTA takes a tile or issues a copy, and each waits expire_ns on a
// barrier phase that nothing can complete.
template <int LEN>
__global__ void __launch_bounds__(LEN, 768 / LEN)
    k_inv_bits_tma(const __grid_constant__ CUtensorMap wmap, uint64_t L, uint64_t m, uint32_t nkeys, uint32_t pairs,
                   const uint32_t *__restrict__ popc, uint32_t *__restrict__ margin_bits, uint64_t *__restrict__ out,
                   uint64_t ostride, TwTab<float> tw, const uint64_t *__restrict__ xkeys, uint64_t xstride,
                   uint32_t *__restrict__ ctl, uint32_t expire_ns) {
    using T = float;
    constexpr int E = 16, COLS = 16;
    static_assert(LEN <= 256 && LEN >= 64, "one tiled copy moves at most 256 rows");
    constexpr uint32_t kTileBytes = LEN * COLS * sizeof(cx<T>);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // a tiled copy's destination must be 128-byte aligned: the launch adds 128 bytes to round up
    unsigned char *base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    cx<T> *stg = reinterpret_cast<cx<T> *>(base);  // staged tile: row a at stg[a * COLS .. +COLS)
    cx<T> *sm = stg + LEN * COLS;                   // exchange buffer of the transform
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t next_tile;
    using word_t = typename BitsWord<COLS>::type;
    const uint32_t col = threadIdx.x % COLS, tq = threadIdx.x / COLS;
    const uint64_t S = L >> ilog2(LEN);
    const uint32_t ncolt = (uint32_t)(S / COLS);
    const uint32_t ntiles = ncolt * pairs;
    const bool aligned = (smem_addr(stg) & 127u) == 0;  // always, given the spare bytes: never copy misaligned
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
        uint32_t t = ntiles;
        if (!aligned) {
            atomicOr(ctl, 2u);
        } else if (expire_ns == 0) {
            t = atomicAdd(ctl + 1, 1u);
            if (t < ntiles) {
                mbar_arrive_expect_tx(&bar, kTileBytes);
                tma_load_2d(stg, &wmap, (int)((t % ncolt) * COLS), (int)((t / ncolt) * LEN), &bar);
            }
        } else if (!mbar_wait(&bar, 0, expire_ns)) {  // test hook: phase 0 never completes
            atomicOr(ctl, 1u);
        }
        next_tile = t;
    }
    __syncthreads();
    uint32_t t = next_tile, phase = 0;
    while (t < ntiles) {
        const bool ok = mbar_wait(&bar, phase);
        phase ^= 1u;
        // also orders this tile's first exchange writes after the last tile's exchange reads
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                atomicOr(ctl, 1u);
                mbar_wait(&bar, phase ^ 1u);  // the copy that ran late: one more bounded wait
            }
            break;
        }
        cx<T> v[E];
#pragma unroll
        for (int s = 0; s < E; ++s) v[s] = stg[idx_e<LEN, E>(tq, s) * COLS + col];
        __syncthreads();  // the staged tile has been read: refill it with the next tile
        if (threadIdx.x == 0) {
            const uint32_t nt = atomicAdd(ctl + 1, 1u);
            if (nt < ntiles) {
                mbar_arrive_expect_tx(&bar, kTileBytes);
                tma_load_2d(stg, &wmap, (int)((nt % ncolt) * COLS), (int)((nt / ncolt) * LEN), &bar);
            }
            next_tile = nt;  // read by every thread after pack_pair_bits' barrier
        }
        const uint32_t pair = t / ncolt;
        const uint64_t u0 = (uint64_t)(t % ncolt) * COLS, u = u0 + col;
        const uint32_t ka = 2 * pair, kb = ka + 1;
        const bool has_b = kb < nkeys;
        twiddle_chain<T, true, E>(v, tw, (uint32_t)(tq * u), (uint32_t)((LEN / E) * u));
        cta_fft<T, LEN, COLS, E, true>(sm, v, tq, col, tw);
        const uint32_t popa = popc[ka], popb = has_b ? popc[kb] : 0u;
        word_t *oa = reinterpret_cast<word_t *>(out + (uint64_t)ka * ostride);
        word_t *ob = reinterpret_cast<word_t *>(out + (uint64_t)kb * ostride);
        pack_pair_bits<T, LEN, COLS, E>(v, tq, col, S, u0, m, m, popa, popb, ka, kb, has_b, oa, ob, margin_bits, xkeys,
                                        xstride);
        t = next_tile;
    }
    if (threadIdx.x == 0 && atomicAdd(ctl + 2, 1u) == gridDim.x - 1) {
        // every CTA has taken its last ticket: reset the counters for the next launch
        atomicExch(ctl + 1, 0u);
        atomicExch(ctl + 2, 0u);
    }
}

}  // namespace pa

// ===========================================================================
// Uneven batch: blocks of different (n, m), each with its own seed, grouped by
// transform length L. Per block the paper's real-valued FFT acceleration
// (Eq. 5-10) carries key and seed in one complex transform, z = x + i*sigma;
// the fused middle pass separates X and V from Z(k) and Z(-k), forms X*V and
// sends two blocks' products through one inverse transform as Y1 + i*Y2.
// ===========================================================================
namespace pa {

// Device-side block descriptor.
struct BlockDev {
    uint64_t n, m;
    const uint64_t *key;   // ceil(n/64) words
    const uint64_t *seed;  // ceil((n+m-1)/64) words
    uint64_t *out;         // ceil(m/64) words
    uint32_t id;           // index of the block in the caller's list (popcount / margin slot)
    uint32_t pad;
};

// Level-1 forward pass of z = x + i*sigma for every block of a class. Grid (S/COLS, blocks).
template <typename T, int LEN, int COLS, int E>
__global__ void __launch_bounds__(COLS * LEN / E, min_blocks(COLS * LEN / E))
    k_fwd_keyseed(const BlockDev *__restrict__ blocks, cx<T> *__restrict__ W, uint64_t L, TwTab<T> tw,
                  uint32_t *__restrict__ popc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    const uint32_t col = threadIdx.x % COLS, tq = threadIdx.x / COLS;
    const uint64_t S = L >> ilog2(LEN);
    const uint64_t u = (uint64_t)blockIdx.x * COLS + col;
    const BlockDev bd = blocks[blockIdx.y];
    const uint64_t n = bd.n, sbits = bd.n + bd.m - 1;
    // stage per row: the CTA's COLS key bits (aligned), COLS seed bits at the rotated
    // position j = a*S + u0 + n - 1 (mod L; the window may wrap past L) and the mask
    // of window positions inside the seed (past it the value is 0, not +-1)
    uint64_t *stage = reinterpret_cast<uint64_t *>(key_stage<T, LEN, COLS>(smem_raw));
    const uint64_t u0 = (uint64_t)blockIdx.x * COLS;
    const uint32_t full = (1u << COLS) - 1u;
    uint32_t ck = 0;  // the CTA's share of the key's popcount P (the CTAs tile every bit once)
    for (uint32_t a = threadIdx.x; a < LEN; a += blockDim.x) {
        const uint64_t t0 = (uint64_t)a * S + u0;
        const uint32_t wk = aligned_bits<COLS>(bd.key, n, t0);
        ck += __popc(wk);
        uint64_t j0 = t0 + n - 1;
        if (j0 >= L) j0 -= L;
        uint32_t ws, inr;
        if (j0 + COLS <= L) {
            ws = bits_at(bd.seed, sbits, j0, COLS);
            inr = j0 >= sbits ? 0u : (sbits - j0 >= COLS ? full : (1u << (sbits - j0)) - 1u);
        } else {  // positions j0 .. L-1, then 0 .. COLS-c1-1 (wrapped)
            const uint32_t c1 = (uint32_t)(L - j0);
            ws = bits_at(bd.seed, sbits, j0, c1) | (bits_at(bd.seed, sbits, 0, COLS - c1) << c1);
            const uint32_t lo = j0 >= sbits ? 0u : (sbits - j0 >= c1 ? (1u << c1) - 1u : (1u << (sbits - j0)) - 1u);
            const uint32_t nw = sbits >= COLS - c1 ? COLS - c1 : (uint32_t)sbits;  // wrapped positions inside the seed
            inr = lo | (((1u << nw) - 1u) << c1);
        }
        stage[a] = (uint64_t)wk | ((uint64_t)ws << 16) | ((uint64_t)inr << 32);
    }
    uint32_t unused = 0u;
    __shared__ uint32_t red[64];
    cta_reduce2<false>(ck, unused, red);  // also publishes the staged rows
    if (threadIdx.x == 0 && ck) atomicAdd(popc + bd.id, ck);
    cx<T> v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const uint64_t w3 = stage[idx_r0<LEN, E>(tq, s)];
        const uint32_t bx = (uint32_t)(w3 >> col) & 1u, bs = (uint32_t)(w3 >> (16 + col)) & 1u;
        const uint32_t inr = (uint32_t)(w3 >> (32 + col)) & 1u;
        v[s] = Arith<T>::mk(bx ? (T)1 : (T)0, inr ? (bs ? (T)-1 : (T)1) : (T)0);
    }
    cta_fft<T, LEN, COLS, E, false>(sm, v, tq, col, tw);
    cx<T> *w = W + (uint64_t)blockIdx.y * L;
    twiddle_chain<T, false, E>(v, tw, (uint32_t)(tq * u), (uint32_t)((LEN / E) * u));
#pragma unroll
    for (int s = 0; s < E; ++s) w[(uint64_t)idx_e<LEN, E>(tq, s) * S + u] = v[s];
}

// Storage row of the frequency low part rho (lgM = log2 of the middle strided
// pass length, 0 for two-level plans): rho = k1 + L1*k2 sits at row k1*M + k2.
__device__ __forceinline__ uint32_t split_row(uint32_t rho, uint32_t lgL1, uint32_t lgM) {
    return ((rho & ((1u << lgL1) - 1u)) << lgM) + (rho >> lgL1);
}

// Fused innermost pass of the uneven batch. CTA (rho, pair): rows rho and
// -rho of blocks 2*pair and 2*pair+1 (if present), one thread group per row.
// Forward transform, Eq. 5-10 split with the mirror bin, X*V/L, then the
// inverse transform of Y1 + i*Y2 written to the pair's slot in Wi.
template <typename T, int LEN, int E>
__global__ void __launch_bounds__(2 * (LEN / E), min_blocks_inner(2 * (LEN / E)))
    k_middle_split(const cx<T> *__restrict__ Wf, cx<T> *__restrict__ Wi, uint64_t L, uint32_t nblocks,
                   uint32_t lgL1, uint32_t lgM, TwTab<T> tw, T inv_L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *smem = reinterpret_cast<cx<T> *>(smem_raw);
    constexpr uint32_t TC = LEN / E;
    constexpr uint32_t SE = smem_elems<LEN, 1>();
    const uint32_t g = threadIdx.x / TC, tq = threadIdx.x % TC;
    const uint32_t R = (uint32_t)(L / LEN);  // rows per block
    const uint32_t rho = blockIdx.x;          // 0 .. R/2
    const uint32_t rho_m = (R - rho) & (R - 1);
    const uint32_t my_rho = g ? rho_m : rho;
    const uint32_t row = split_row(my_rho, lgL1, lgM);
    const bool self_paired = rho == rho_m;
    cx<T> *sm = smem + g * SE;                          // this group's transform scratch
    const cx<T> *sm_other = smem + (self_paired ? g : 1u - g) * SE;  // where the mirror row's spectrum sits
    const uint32_t b1 = 2 * blockIdx.y, b2 = b1 + 1;
    const bool has2 = b2 < nblocks;
    cx<T> y[E];
#pragma unroll
    for (int s = 0; s < E; ++s) y[s] = Arith<T>::mk((T)0, (T)0);
    for (int which = 0; which < (has2 ? 2 : 1); ++which) {
        const cx<T> *wt = Wf + (uint64_t)(which ? b2 : b1) * L + (uint64_t)row * LEN + tq;
        cx<T> v[E];
        __syncthreads();  // previous use of the scratch is finished
        if constexpr (Plan<LEN, E>::RO == 1) {
#pragma unroll
            for (int s = 0; s < E; ++s) v[s] = wt[idx_r0<LEN, E>(0, s)];
            cta_fft<T, LEN, 1, E, false>(sm, v, tq, 0, tw);
        } else {
            cta_fft_fwd_odd<T, LEN, E>(sm, v, tq, tw, [&](uint32_t o) { return wt[o]; });
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < E; ++s) sm[sidx<1>(idx_e<LEN, E>(tq, s), 0)] = v[s];
        __syncthreads();
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const uint32_t p = idx_e<LEN, E>(tq, s);
            // mirror of position p: -p mod LEN in the row of the zero frequency low part, else LEN-1-p
            const uint32_t pm = (my_rho == 0) ? (p == 0 ? 0u : (uint32_t)LEN - p) : ((uint32_t)LEN - 1u - p);
            const cx<T> z = v[s], zm = sm_other[sidx<1>(pm, 0)];
            // Eq. 7-10: X = (Z(k) + conj Z(-k)) / 2, V = (Z(k) - conj Z(-k)) / (2i)
            const cx<T> X = Arith<T>::mk((z.x + zm.x) * (T)0.5, (z.y - zm.y) * (T)0.5);
            const cx<T> V = Arith<T>::mk((z.y + zm.y) * (T)0.5, (zm.x - z.x) * (T)0.5);
            cx<T> Y = Arith<T>::mul(X, V);
            Y.x *= inv_L;
            Y.y *= inv_L;
            if (which == 0) {
                y[s] = Y;
            } else {  // y += i * Y2
                y[s].x -= Y.y;
                y[s].y += Y.x;
            }
        }
    }
    __syncthreads();
    cx<T> *wot = Wi + (uint64_t)blockIdx.y * L + (uint64_t)row * LEN + tq;
    const bool store = !(self_paired && g == 1);  // a self-paired row is written once
    if constexpr (Plan<LEN, E>::RO == 1) {
        cta_fft<T, LEN, 1, E, true>(sm, y, tq, 0, tw);
        if (!store) return;
#pragma unroll
        for (int s = 0; s < E; ++s) wot[idx_r0<LEN, E>(0, s)] = y[s];
    } else {
        cta_fft_inv_odd<T, LEN, E>(sm, y, tq, tw, [&](uint32_t o, cx<T> x) {
            if (store) wot[o] = x;
        });
    }
}

// Fused innermost pass of a single key in a half-length transform (the real-input
// form of the convolution theorem; paper Eq. 5-10 give the same split for a key and
// a seed). The slot holds Z = FFT_N(z), z[t] = x[2t] + i x[2t+1], N = L/2. With the
// mirror bin Z' = Z[N-k]: E_x = (Z + conj Z')/2 and O_x = (Z - conj Z')/(2i) are the
// spectra of the even and odd key bits, and with the seed tables (per bin, times 1/N)
// Es = E_s, Os = O_s and Bp = w_N^k O_s of the seed's even/odd spectra, the product
// Y = S X of the length-L transforms is, in even/odd form,
//     E_y = Es E_x + Bp O_x,   O_y = Es O_x + Os E_x,
// and the inverse transform of E_y + i O_y returns y[2t] + i y[2t+1].
// CTA (rho, slot): rows rho and -rho (one thread group each), as in k_middle_split.
// MODE 1 builds the tables from the seed slot instead (forward transform and split only).
template <typename T, int LEN, int E, int MODE>
__global__ void __launch_bounds__(2 * (LEN / E), min_blocks_inner(2 * (LEN / E)))
    k_middle_real(cx<T> *__restrict__ W, cx<T> *__restrict__ tabs, uint64_t N, uint32_t lgL1, uint32_t lgM,
                  TwTab<T> tw, T scale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *smem = reinterpret_cast<cx<T> *>(smem_raw);
    constexpr uint32_t TC = LEN / E;
    constexpr uint32_t SE = smem_elems<LEN, 1>();
    const uint32_t g = threadIdx.x / TC, tq = threadIdx.x % TC;
    const uint32_t R = (uint32_t)(N / LEN);  // rows
    const uint32_t rho = blockIdx.x;          // 0 .. R/2
    const uint32_t rho_m = (R - rho) & (R - 1);
    const uint32_t my_rho = g ? rho_m : rho;
    const uint32_t row = split_row(my_rho, lgL1, lgM);
    const bool self_paired = rho == rho_m;
    cx<T> *sm = smem + g * SE;
    const cx<T> *sm_other = smem + (self_paired ? g : 1u - g) * SE;
    cx<T> *wt = W + (uint64_t)blockIdx.y * N + (uint64_t)row * LEN + tq;
    cx<T> v[E];
    if constexpr (Plan<LEN, E>::RO == 1) {
#pragma unroll
        for (int s = 0; s < E; ++s) v[s] = wt[idx_r0<LEN, E>(0, s)];
        cta_fft<T, LEN, 1, E, false>(sm, v, tq, 0, tw);
    } else {
        cta_fft_fwd_odd<T, LEN, E>(sm, v, tq, tw, [&](uint32_t o) { return wt[o]; });
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < E; ++s) sm[sidx<1>(idx_e<LEN, E>(tq, s), 0)] = v[s];
    __syncthreads();
    const cx<T> *Es = tabs, *Os = tabs + N, *Bp = tabs + 2 * N;
    const bool write_tab = !(self_paired && g == 1);
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const uint32_t p = idx_e<LEN, E>(tq, s);
        // mirror of position p: -p mod LEN in the row of the zero frequency low part, else LEN-1-p
        const uint32_t pm = (my_rho == 0) ? (p == 0 ? 0u : (uint32_t)LEN - p) : ((uint32_t)LEN - 1u - p);
        const cx<T> z = v[s], zm = sm_other[sidx<1>(pm, 0)];
        const cx<T> ex = Arith<T>::mk((z.x + zm.x) * (T)0.5, (z.y - zm.y) * (T)0.5);
        const cx<T> ox = Arith<T>::mk((z.y + zm.y) * (T)0.5, (zm.x - z.x) * (T)0.5);
        const uint64_t e = (uint64_t)row * LEN + p;
        if constexpr (MODE == 1) {
            if (write_tab) {
                const cx<T> es = Arith<T>::mk(ex.x * scale, ex.y * scale);
                const cx<T> os = Arith<T>::mk(ox.x * scale, ox.y * scale);
                // frequency of this bin: low part from the strided passes, high part p
                const uint32_t k = my_rho + R * p;
                tabs[e] = es;
                tabs[N + e] = os;
                tabs[2 * N + e] = Arith<T>::mul(Arith<T>::template omega<false>(tw, k), os);
            }
        } else {
            const cx<T> es = Es[e], os = Os[e], bp = Bp[e];
            const cx<T> ey = Arith<T>::add(Arith<T>::mul(es, ex), Arith<T>::mul(bp, ox));
            const cx<T> oy = Arith<T>::add(Arith<T>::mul(es, ox), Arith<T>::mul(os, ex));
            v[s] = Arith<T>::mk(ey.x - oy.y, ey.y + oy.x);  // E_y + i O_y
        }
    }
    if constexpr (MODE == 0) {
        __syncthreads();  // the mirror reads of both groups are done
        const bool store = !(self_paired && g == 1);  // a self-paired row is written once
        if constexpr (Plan<LEN, E>::RO == 1) {
            cta_fft<T, LEN, 1, E, true>(sm, v, tq, 0, tw);
            if (!store) return;
#pragma unroll
            for (int s = 0; s < E; ++s) wt[idx_r0<LEN, E>(0, s)] = v[s];
        } else {
            cta_fft_inv_odd<T, LEN, E>(sm, v, tq, tw, [&](uint32_t o, cx<T> x) {
                if (store) wt[o] = x;
            });
        }
    }
}

// Level-1 inverse pass with bit output for pairs of blocks (real part: block
// 2p, imaginary part: block 2p+1), each with its own m and output pointer.
template <typename T, int LEN, int COLS, int E>
__global__ void __launch_bounds__(COLS * LEN / E, min_blocks(COLS * LEN / E))
    k_inv_bits_blocks(const cx<T> *__restrict__ W, uint64_t L, const BlockDev *__restrict__ blocks, uint32_t nblocks,
                      const uint32_t *__restrict__ popc, uint32_t *__restrict__ margin_bits, TwTab<T> tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    using word_t = typename BitsWord<COLS>::type;
    const uint32_t col = threadIdx.x % COLS, tq = threadIdx.x / COLS;
    const uint64_t S = L >> ilog2(LEN);
    const uint64_t u0 = (uint64_t)blockIdx.x * COLS;
    const uint64_t u = u0 + col;
    const uint32_t ia = 2 * blockIdx.y, ib = ia + 1;
    const bool has_b = ib < nblocks;
    const BlockDev ba_ = blocks[ia];
    const BlockDev bb_ = blocks[has_b ? ib : ia];
    const cx<T> *w = W + (uint64_t)blockIdx.y * L;
    cx<T> v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = w[(uint64_t)idx_e<LEN, E>(tq, s) * S + u];
    twiddle_chain<T, true, E>(v, tw, (uint32_t)(tq * u), (uint32_t)((LEN / E) * u));
    cta_fft<T, LEN, COLS, E, true>(sm, v, tq, col, tw);
    const uint32_t popa = popc[ba_.id];
    const uint32_t popb = has_b ? popc[bb_.id] : 0u;
    word_t *oa = reinterpret_cast<word_t *>(ba_.out);
    word_t *ob = reinterpret_cast<word_t *>(bb_.out);
    // each block decoded with its own m: the real part is block 2p, the imaginary part block 2p+1
    pack_pair_bits<T, LEN, COLS, E>(v, tq, col, S, u0, ba_.m, bb_.m, popa, popb, ba_.id, bb_.id, has_b, oa, ob,
                                    margin_bits, nullptr, 0);
}

}  // namespace pa

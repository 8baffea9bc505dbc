// fft_core.cuh -- device building blocks of the FFT passes.
//
// The hash is evaluated through the convolution theorem (paper Eq. 4). A long
// transform of length L is split into passes of short transforms in the spirit
// of the paper's Algorithm 1 (row FFTs, twiddle factors W[i*j], column FFTs).
// Unlike Algorithm 1 the passes never transpose: each forward pass is a
// decimation-in-frequency step that leaves the spectrum in digit-reversed
// order, the pointwise product does not care about order (the seed spectrum
// is stored in the same order), and the inverse passes undo the steps in
// reverse so the convolution comes out in natural order. This is the GPU form
// of Algorithm 2's observation that the spectrum's order is irrelevant to PA,
// without Algorithm 2's permutation of the final key.
//
// Inside a CTA a short transform of length LEN runs as a Stockham autosort FFT:
// every thread holds E complex values in registers, does radix-R butterflies
// (R <= E) in registers, and exchanges through shared memory between stages.
// A CTA works on COLS transforms at once, interleaved column-wise in shared
// memory, so that a warp's global accesses touch COLS consecutive elements.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace pa {

// Element arithmetic of the transforms. Arith<float> / Arith<double> work on
// complex numbers (x = real, y = imaginary); Arith<Zp> (zp.cuh) on residues
// modulo the prime p = 2^64 - 2^32 + 1. The FFT engine below only uses add,
// sub, mul, the in-register roots rot32 and the table twiddles omega.
template <typename T> struct Arith;
template <typename T> using cx = typename Arith<T>::E;

// cos(pi*j/16), j = 0..8, to 20 significant digits.
__host__ __device__ constexpr double cos_pi16(int j) {
    return j == 0   ? 1.0
           : j == 1 ? 0.98078528040323044913
           : j == 2 ? 0.92387953251128675613
           : j == 3 ? 0.83146961230254523708
           : j == 4 ? 0.70710678118654752440
           : j == 5 ? 0.55557023301960222474
           : j == 6 ? 0.38268343236508977173
           : j == 7 ? 0.19509032201612826785
                    : 0.0;
}
// cos and sin of 2*pi*j/32 for 0 <= j < 16.
__host__ __device__ constexpr double cos32(int j) { return j <= 8 ? cos_pi16(j) : -cos_pi16(16 - j); }
__host__ __device__ constexpr double sin32(int j) { return j <= 8 ? cos_pi16(8 - j) : cos_pi16(j - 8); }

// Twiddle table pair for the length-L transform root w_L: w_L^e = hi[e >> B] * lo[e & (2^B-1)].
// Complex roots are exp(-2*pi*i/L), computed in double precision on the host and rounded to T.
template <typename T> struct TwTab {
    const cx<T> *hi;
    const cx<T> *lo;
    uint32_t B;    // split position
    uint32_t lgL;  // log2 L
};

template <typename T> struct ComplexArith {
    using E = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    static __device__ __forceinline__ E mk(T x, T y) { E r; r.x = x; r.y = y; return r; }
    static __device__ __forceinline__ E add(E a, E b) { return mk(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ E sub(E a, E b) { return mk(a.x - b.x, a.y - b.y); }
    static __device__ __forceinline__ E mul(E a, E b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
    // x * w^j with w = exp(-2*pi*i/32) (forward) or its conjugate (inverse). j is a
    // compile-time constant after unrolling, so the branches fold away.
    template <bool INV> static __device__ __forceinline__ E rot32(E x, int j) {
        if (j == 0) return x;
        if (j == 8) return INV ? mk(-x.y, x.x) : mk(x.y, -x.x);
        const T c = (T)cos32(j);
        const T s = INV ? (T)sin32(j) : -(T)sin32(j);
        return mk(x.x * c - x.y * s, x.x * s + x.y * c);
    }
    template <bool INV> static __device__ __forceinline__ E omega(const TwTab<T> &t, uint32_t e) {
        E a = __ldg(t.hi + (e >> t.B));
        E b = __ldg(t.lo + (e & ((1u << t.B) - 1u)));
        E w = mul(a, b);
        if (INV) w.y = -w.y;
        return w;
    }
};
template <> struct Arith<float> : ComplexArith<float> {};
template <> struct Arith<double> : ComplexArith<double> {};

}  // namespace pa

#include "zp.cuh"

namespace pa {

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }
__host__ __device__ constexpr int bitrev(int v, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
    return r;
}

// In-register DFT of R = 2^s <= 32 values, natural order in and out:
// radix-2 decimation in frequency followed by a register renaming.
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft(cx<T> *v) {
    static_assert(R >= 1 && R <= 32 && (R & (R - 1)) == 0, "radix must be a power of two <= 32");
    if constexpr (R > 1) {
#pragma unroll
        for (int len = R; len >= 2; len >>= 1) {
#pragma unroll
            for (int b = 0; b < R; b += len) {
#pragma unroll
                for (int j = 0; j < len / 2; ++j) {
                    cx<T> a = v[b + j], c = v[b + j + len / 2];
                    v[b + j] = Arith<T>::add(a, c);
                    v[b + j + len / 2] = Arith<T>::template rot32<INV>(Arith<T>::sub(a, c), j * (32 / len));
                }
            }
        }
        cx<T> t[R];
#pragma unroll
        for (int k = 0; k < R; ++k) t[k] = v[bitrev(k, ilog2(R))];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = t[k];
    }
}

// v[r] *= w_L^{e0 + r*de} for r = 0..N-1: two table lookups, then a chain of
// complex products (relative error grows by about one rounding per step).
template <typename T, bool INV, int N>
__device__ __forceinline__ void twiddle_chain(cx<T> *v, const TwTab<T> &tw, uint32_t e0, uint32_t de) {
    const cx<T> g = Arith<T>::template omega<INV>(tw, de);
    cx<T> w = (e0 == 0u) ? g : Arith<T>::template omega<INV>(tw, e0 + de);
    if (e0 != 0u) v[0] = Arith<T>::mul(v[0], Arith<T>::template omega<INV>(tw, e0));
#pragma unroll
    for (int r = 1; r < N; ++r) {
        v[r] = Arith<T>::mul(v[r], w);
        if (r + 1 < N) w = Arith<T>::mul(w, g);
    }
}

// Shared-memory slot of element a of column col (COLS columns interleaved),
// skewed by one slot every 16 to keep Stockham's strided writes conflict-free.
template <int COLS>
__device__ __forceinline__ uint32_t sidx(uint32_t a, uint32_t col) {
    uint32_t i = a * COLS + col;
    return i + (i >> 4);
}
template <int LEN, int COLS>
constexpr uint32_t smem_elems() { return (uint32_t)LEN * COLS + ((uint32_t)LEN * COLS >> 4) + 1; }

// Stage plan of a Stockham FFT of length LEN with E values per thread:
// q stages; the forward transform uses radices [R0, E, ..., E], the inverse
// [E, ..., E, R0], so the forward's output distribution over threads equals
// the inverse's input distribution and the two chain in registers.
template <int LEN, int E> struct Plan {
    static constexpr int k = ilog2(LEN), e = ilog2(E);
    static constexpr int q = (k + e - 1) / e;
    static constexpr int r0 = 1 << (k - (q - 1) * e);
    static constexpr int TC = LEN / E;  // threads per column
    static_assert(q >= 2, "LEN must exceed E");
    static_assert((1 << k) == LEN && (1 << e) == E, "powers of two only");
};

// Index of the element that register slot s of thread tq holds at the start
// (first-stage input) and at the end (last-stage output) of a transform.
//   forward start / inverse end:  slot b*R0 + r  ->  tq + b*TC + r*(LEN/R0)
//   forward end / inverse start:  slot r         ->  tq + r*TC
template <int LEN, int E>
__device__ __forceinline__ uint32_t idx_r0(uint32_t tq, int s) {
    using P = Plan<LEN, E>;
    return tq + (uint32_t)(s / P::r0) * P::TC + (uint32_t)(s % P::r0) * (LEN / P::r0);
}
template <int LEN, int E>
__device__ __forceinline__ uint32_t idx_e(uint32_t tq, int s) {
    return tq + (uint32_t)s * (LEN / E);
}

// One Stockham stage of radix R at span p, from registers (already loaded
// with this stage's inputs) to shared memory. Thread tq handles the E/R
// butterfly groups i = tq + b*TC; group i reads elements i + r*LEN/R,
// multiplies by w_{R p}^{r k} (k = i mod p), transforms, and writes element
// (i - k)*R + k + r*p.
template <typename T, int LEN, int COLS, int E, int R, bool INV>
__device__ __forceinline__ void stage_to_smem(cx<T> *sm, cx<T> *v, uint32_t tq, uint32_t col, uint32_t p,
                                              const TwTab<T> &tw) {
    constexpr int TC = LEN / E;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        const uint32_t i = tq + (uint32_t)b * TC;
        const uint32_t k = i & (p - 1);
        if (p > 1) twiddle_chain<T, INV, R>(v + b * R, tw, 0u, k << (tw.lgL - ilog2(R) - (31 - __clz(p))));
        dft<T, R, INV>(v + b * R);
        const uint32_t base = (i - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) sm[sidx<COLS>(base + (uint32_t)r * p, col)] = v[b * R + r];
    }
}

// Load a stage's inputs from shared memory: group i = tq + b*TC, elements i + r*LEN/R.
template <typename T, int LEN, int COLS, int E, int R>
__device__ __forceinline__ void load_from_smem(const cx<T> *sm, cx<T> *v, uint32_t tq, uint32_t col) {
    constexpr int TC = LEN / E;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        const uint32_t i = tq + (uint32_t)b * TC;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = sm[sidx<COLS>(i + (uint32_t)r * (LEN / R), col)];
    }
}

// Last stage: twiddle + DFT in registers, results stay in registers.
template <typename T, int LEN, int E, int R, bool INV>
__device__ __forceinline__ void stage_in_regs(cx<T> *v, uint32_t tq, uint32_t p, const TwTab<T> &tw) {
    constexpr int TC = LEN / E;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        const uint32_t i = tq + (uint32_t)b * TC;
        const uint32_t k = i & (p - 1);
        if (p > 1) twiddle_chain<T, INV, R>(v + b * R, tw, 0u, k << (tw.lgL - ilog2(R) - (31 - __clz(p))));
        dft<T, R, INV>(v + b * R);
    }
}

// Full transform of length LEN on COLS interleaved columns. On entry v holds
// the first-stage inputs (forward: idx_r0 layout; inverse: idx_e layout); on
// exit v holds the outputs (forward: idx_e layout; inverse: idx_r0 layout).
// The caller must __syncthreads() before the call if shared memory is still
// being read from a previous transform.
template <typename T, int LEN, int COLS, int E, bool INV>
__device__ __forceinline__ void cta_fft(cx<T> *sm, cx<T> *v, uint32_t tq, uint32_t col, const TwTab<T> &tw) {
    using P = Plan<LEN, E>;
    // radix of stage s: forward [R0, E, ..., E], inverse [E, ..., E, R0]
    uint32_t p = 1;
    if constexpr (!INV) {
        stage_to_smem<T, LEN, COLS, E, P::r0, INV>(sm, v, tq, col, p, tw);
        p *= P::r0;
#pragma unroll
        for (int s = 1; s < P::q - 1; ++s) {
            __syncthreads();
            load_from_smem<T, LEN, COLS, E, E>(sm, v, tq, col);
            __syncthreads();
            stage_to_smem<T, LEN, COLS, E, E, INV>(sm, v, tq, col, p, tw);
            p *= E;
        }
        __syncthreads();
        load_from_smem<T, LEN, COLS, E, E>(sm, v, tq, col);
        stage_in_regs<T, LEN, E, E, INV>(v, tq, p, tw);
    } else {
        stage_to_smem<T, LEN, COLS, E, E, INV>(sm, v, tq, col, p, tw);
        p *= E;
#pragma unroll
        for (int s = 1; s < P::q - 1; ++s) {
            __syncthreads();
            load_from_smem<T, LEN, COLS, E, E>(sm, v, tq, col);
            __syncthreads();
            stage_to_smem<T, LEN, COLS, E, E, INV>(sm, v, tq, col, p, tw);
            p *= E;
        }
        __syncthreads();
        load_from_smem<T, LEN, COLS, E, P::r0>(sm, v, tq, col);
        stage_in_regs<T, LEN, E, P::r0, INV>(v, tq, p, tw);
    }
}

}  // namespace pa

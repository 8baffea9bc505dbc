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

// In-register DFT of RO = 3, 5 or 9 complex values (odd factors of smooth
// transform lengths), natural order in and out. Forward roots w_R = exp(-2 pi i / R).
// Constants: cos/sin of 2 pi j / R to 20 significant digits.
template <typename T, bool INV>
__device__ __forceinline__ void dft3(cx<T> &x0, cx<T> &x1, cx<T> &x2) {
    constexpr T s3 = (T)0.86602540378443864676;  // sin(2 pi / 3)
    const cx<T> a = Arith<T>::add(x1, x2), b = Arith<T>::sub(x1, x2);
    const cx<T> c = Arith<T>::mk(x0.x - (T)0.5 * a.x, x0.y - (T)0.5 * a.y);
    // forward: y1 = c - i s3 b, y2 = c + i s3 b (inverse swaps the signs)
    const T sb_x = (INV ? -s3 : s3) * b.x, sb_y = (INV ? -s3 : s3) * b.y;
    x0 = Arith<T>::add(x0, a);
    x1 = Arith<T>::mk(c.x + sb_y, c.y - sb_x);
    x2 = Arith<T>::mk(c.x - sb_y, c.y + sb_x);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft5(cx<T> *x) {
    constexpr T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
    constexpr T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
    const cx<T> a1 = Arith<T>::add(x[1], x[4]), b1 = Arith<T>::sub(x[1], x[4]);
    const cx<T> a2 = Arith<T>::add(x[2], x[3]), b2 = Arith<T>::sub(x[2], x[3]);
    const cx<T> x0 = x[0];
    // real-coefficient parts
    const cx<T> p1 = Arith<T>::mk(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
    const cx<T> p2 = Arith<T>::mk(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
    // q1 = s1 b1 + s2 b2, q2 = s2 b1 - s1 b2; y1 = p1 - i q1, y4 = p1 + i q1, y2 = p2 - i q2, y3 = p2 + i q2
    T q1x = s1 * b1.x + s2 * b2.x, q1y = s1 * b1.y + s2 * b2.y;
    T q2x = s2 * b1.x - s1 * b2.x, q2y = s2 * b1.y - s1 * b2.y;
    if (INV) { q1x = -q1x; q1y = -q1y; q2x = -q2x; q2y = -q2y; }
    x[0] = Arith<T>::add(x0, Arith<T>::add(a1, a2));
    x[1] = Arith<T>::mk(p1.x + q1y, p1.y - q1x);
    x[4] = Arith<T>::mk(p1.x - q1y, p1.y + q1x);
    x[2] = Arith<T>::mk(p2.x + q2y, p2.y - q2x);
    x[3] = Arith<T>::mk(p2.x - q2y, p2.y + q2x);
}

// x * w9^j for the radix-9 internal twiddles (j in 1, 2, 4).
template <typename T, bool INV>
__device__ __forceinline__ cx<T> rot9(cx<T> x, int j) {
    const T c = j == 1 ? (T)0.76604444311897803520 : j == 2 ? (T)0.17364817766693034885 : (T)-0.93969262078590838405;
    const T sn = j == 1 ? (T)0.64278760968653932632 : j == 2 ? (T)0.98480775301220805936 : (T)0.34202014332566873304;
    const T s = INV ? sn : -sn;
    return Arith<T>::mk(x.x * c - x.y * s, x.x * s + x.y * c);
}

template <typename T, int RO, bool INV>
__device__ __forceinline__ void dft_odd(cx<T> *x) {
    if constexpr (RO == 3) {
        dft3<T, INV>(x[0], x[1], x[2]);
    } else if constexpr (RO == 5) {
        dft5<T, INV>(x);
    } else {
        static_assert(RO == 9, "odd radix must be 3, 5 or 9");
        // 9 = 3 x 3: x[3m + r] -> DFT3 over m for each r, twiddle w9^{r k1}, DFT3 over r; X[k1 + 3 k2]
        cx<T> a[9];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            cx<T> u0 = x[r], u1 = x[3 + r], u2 = x[6 + r];
            dft3<T, INV>(u0, u1, u2);
            a[3 * r + 0] = u0;  // k1 = 0
            a[3 * r + 1] = r ? rot9<T, INV>(u1, r) : u1;
            a[3 * r + 2] = r ? rot9<T, INV>(u2, 2 * r) : u2;
        }
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            cx<T> v0 = a[k1], v1 = a[3 + k1], v2 = a[6 + k1];
            dft3<T, INV>(v0, v1, v2);
            x[k1] = v0;
            x[k1 + 3] = v1;
            x[k1 + 6] = v2;
        }
    }
}

// cos and sin of 2 pi a / b in double precision at compile time: the angle is
// reduced to [0, pi/4] by the symmetries of the circle, then summed as a Taylor
// series (terms up to x^27 / 27!, below 1e-30 for |x| <= pi/4).
__host__ __device__ constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k <= 13; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k <= 13; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
constexpr double kPi = 3.14159265358979323846264338327950288;
// cos (SIN = false) or sin (SIN = true) of 2 pi a / b for 0 <= a < b: with 4a = q b + r,
// the angle is q pi/2 + psi, psi = (pi/2) r / b; psi above pi/4 is taken as
// pi/2 - (pi/2)(b - r)/b so the series always runs on [0, pi/4].
__host__ __device__ constexpr double trig_frac(int a, int b, bool want_sin) {
    const int q = (4 * a) / b, r = (4 * a) % b;
    const bool high = 2 * r > b;
    const double psi = (kPi / 2.0) * (double)(high ? b - r : r) / (double)b;
    const double c0 = high ? taylor_sin(psi) : taylor_cos(psi);
    const double s0 = high ? taylor_cos(psi) : taylor_sin(psi);
    // rotate (c0, s0) by q quarter turns
    const double c = q == 0 ? c0 : q == 1 ? -s0 : q == 2 ? -c0 : s0;
    const double sn = q == 0 ? s0 : q == 1 ? c0 : q == 2 ? -s0 : -c0;
    return want_sin ? sn : c;
}
__host__ __device__ constexpr double cos_frac(int a, int b) { return trig_frac(a, b, false); }
__host__ __device__ constexpr double sin_frac(int a, int b) { return trig_frac(a, b, true); }

// x * w_N^J (forward root w_N = exp(-2 pi i / N); the inverse uses the conjugate),
// with the half and quarter turns done exactly.
template <typename T, int N, int J, bool INV>
__device__ __forceinline__ cx<T> rot_const(cx<T> x) {
    constexpr int j = J % N;
    if constexpr (j == 0) {
        return x;
    } else if constexpr (2 * j == N) {
        return Arith<T>::mk(-x.x, -x.y);
    } else if constexpr (4 * j == N) {
        return INV ? Arith<T>::mk(-x.y, x.x) : Arith<T>::mk(x.y, -x.x);
    } else if constexpr (4 * j == 3 * N) {
        return INV ? Arith<T>::mk(x.y, -x.x) : Arith<T>::mk(-x.y, x.x);
    } else {
        constexpr T c = (T)cos_frac(j, N);
        constexpr T sn = (T)sin_frac(j, N);
        constexpr T s = INV ? sn : -sn;
        return Arith<T>::mk(x.x * c - x.y * s, x.x * s + x.y * c);
    }
}

// a[n2 * RO + k1] *= w_{RO R0}^{n2 k1} for n2 >= N2, k1 >= K1 (compile-time indices).
template <typename T, int RO, int R0, int N2, int K1, bool INV>
__device__ __forceinline__ void comp_twiddle_row(cx<T> *a) {
    if constexpr (K1 < RO) {
        a[N2 * RO + K1] = rot_const<T, RO * R0, N2 * K1, INV>(a[N2 * RO + K1]);
        comp_twiddle_row<T, RO, R0, N2, K1 + 1, INV>(a);
    }
}
template <typename T, int RO, int R0, int N2, bool INV>
__device__ __forceinline__ void comp_twiddles(cx<T> *a) {
    if constexpr (N2 < R0) {
        comp_twiddle_row<T, RO, R0, N2, 1, INV>(a);
        comp_twiddles<T, RO, R0, N2 + 1, INV>(a);
    }
}

template <typename T, int R, bool INV> __device__ __forceinline__ void dft(cx<T> *v);

// In-register DFT of RC = RO * R0 values (RO in {3, 5, 9}, R0 a power of two),
// natural order in and out, by one Cooley-Tukey step: with n = R0 n1 + n2 and
// k = k1 + RO k2, X[k] = sum_n2 w_R0^{n2 k2} w_RC^{n2 k1} sum_n1 w_RO^{n1 k1} x[n].
template <typename T, int RO, int R0, bool INV>
__device__ __forceinline__ void dft_comp(cx<T> *x) {
    if constexpr (R0 == 1) {
        dft_odd<T, RO, INV>(x);
    } else {
        cx<T> a[RO * R0];  // a[n2 * RO + k1]
#pragma unroll
        for (int n2 = 0; n2 < R0; ++n2) {
            cx<T> u[RO];
#pragma unroll
            for (int n1 = 0; n1 < RO; ++n1) u[n1] = x[R0 * n1 + n2];
            dft_odd<T, RO, INV>(u);
#pragma unroll
            for (int k1 = 0; k1 < RO; ++k1) a[n2 * RO + k1] = u[k1];
        }
        comp_twiddles<T, RO, R0, 1, INV>(a);
#pragma unroll
        for (int k1 = 0; k1 < RO; ++k1) {
            cx<T> w[R0];
#pragma unroll
            for (int n2 = 0; n2 < R0; ++n2) w[n2] = a[n2 * RO + k1];
            dft<T, R0, INV>(w);
#pragma unroll
            for (int k2 = 0; k2 < R0; ++k2) x[k1 + RO * k2] = w[k2];
        }
    }
}

// Twiddle table pair for the length-L transform root w_L: w_L^e = hi[e >> B] * lo[e & (2^B-1)].
// Complex roots are exp(-2*pi*i/L), computed in double precision on the host and rounded to T.
template <typename T> struct TwTab {
    const cx<T> *hi;
    const cx<T> *lo;
    uint32_t B;    // split position
    uint32_t lgL;  // log2 L
    // In-CTA stage twiddles: fine[j] = w_F^j, where F (a divisor of L) is a
    // multiple of every pass length of the plan.
    const cx<T> *fine;
    uint32_t F;
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
    template <bool INV> static __device__ __forceinline__ E fine(const TwTab<T> &t, uint32_t e) {
        E w = __ldg(t.fine + e);
        if (INV) w.y = -w.y;
        return w;
    }
    template <bool INV> static __device__ __forceinline__ E omega(const TwTab<T> &t, uint32_t e) {
        E a = __ldg(t.hi + (e >> t.B));
        E b = __ldg(t.lo + (e & ((1u << t.B) - 1u)));
        E w = mul(a, b);
        if (INV) w.y = -w.y;
        return w;
    }
};
// FP32 complex add/sub as one packed f32x2 instruction each (sm_100+ packed FP32):
// the (re, im) pair sits in one 64-bit register pair.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
// d = a * b + c on both lanes of an f32x2 pair (one packed instruction).
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
template <> struct Arith<float> : ComplexArith<float> {
    static __device__ __forceinline__ E add(E a, E b) { return f2_add(a, b); }
    static __device__ __forceinline__ E sub(E a, E b) { return f2_sub(a, b); }
};
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

// v[r] *= w_F^{r*step} for r = 1..N-1 (the stage twiddle w_{R p}^{r k} is
// w_F^{r k F/(R p)}). CHAIN = true (used by every pass): one table load, then a
// chain of products -- fewest loads and registers, measured faster than one
// load per value in every pass but the last inverse one, where it is even.
// CHAIN = false: one table load per value.
template <typename T, bool INV, int N, bool CHAIN = true>
__device__ __forceinline__ void stage_twiddles(cx<T> *v, const TwTab<T> &tw, uint32_t step) {
    if constexpr (CHAIN) {
        const cx<T> g = Arith<T>::template fine<INV>(tw, step);
        cx<T> w = g;
#pragma unroll
        for (int r = 1; r < N; ++r) {
            v[r] = Arith<T>::mul(v[r], w);
            if (r + 1 < N) w = Arith<T>::mul(w, g);
        }
    } else {
        uint32_t e = step;
#pragma unroll
        for (int r = 1; r < N; ++r) {
            v[r] = Arith<T>::mul(v[r], Arith<T>::template fine<INV>(tw, e));
            e += step;
        }
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
__host__ __device__ constexpr int odd_part(int v) { return (v & 1) ? v : odd_part(v >> 1); }
constexpr int kMaxCompositeRadix = 24;
__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Stage plan of a Stockham FFT of length LEN = RO * 2^k2 (RO odd: 1, 3, 5 or 9)
// with E values per thread (TC = LEN / E threads per column). Radices:
//   forward  [RO], R0, E, ..., E        inverse  E, ..., E, R0, [RO]
// so the forward's output distribution over threads equals the inverse's input
// distribution (the two chain in registers). An odd stage exists only in
// transforms that read their input from, and write their output to, memory
// (the innermost pass), because its E / RO groups per thread do not divide.
template <int LEN, int E> struct Plan {
    static constexpr int RO = odd_part(LEN);
    static constexpr int K2 = LEN / RO;
    static constexpr int k = ilog2(K2), e = ilog2(E);
    static constexpr int q = (k + e - 1) / e;  // power-of-two stages
    static constexpr int r0 = 1 << (k - (q - 1) * e);
    static constexpr int TC = LEN / E;  // threads per column
    // The odd stage absorbs the radix-r0 stage when r0 < E and the composite radix
    // RO * r0 stays within a register budget: stages [RO * r0], E, ..., E.
    static constexpr bool FOLD = RO > 1 && r0 < E && RO * r0 <= kMaxCompositeRadix;
    static constexpr int R0C = FOLD ? r0 : 1;  // power-of-two factor of the odd stage
    static constexpr int RC = RO * R0C;        // radix of the odd stage
    static_assert(RO == 1 || RO == 3 || RO == 5 || RO == 9, "odd factor must be 1, 3, 5 or 9");
    static_assert(RO > 1 || q >= 2, "LEN must exceed E");
    static_assert((1 << k) == K2 && (1 << e) == E && K2 >= E, "power-of-two part must be >= E");
};

// Index of the element that register slot s of thread tq holds at the start
// (first-stage input) and at the end (last-stage output) of a transform.
//   forward start / inverse end:  slot b*R0 + r  ->  tq + b*TC + r*(LEN/R0)   (RO == 1)
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

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

// Shared-memory slot of element a of a contiguous row (one column) at a stage
// boundary of span SPAN (the reading stage's span: the writing stage has P * R = SPAN).
// Power-of-two spans (every boundary of a power-of-two row, and the inverse
// transform's) use the skew of sidx. A row with an odd stage of radix RC writes
// with strides RC and R * RC in the forward transform, which that skew leaves
// 2-4-way bank conflicted; those boundaries (spans divisible by RC) pad one slot
// every lcm(RC, W) elements instead (W = elements per 128 bytes), and the first one
// keeps the plain index when RC is odd (an odd stride is conflict-free as it is).
template <typename T, int LEN, int E, int SPAN>
__device__ __forceinline__ uint32_t ridx(uint32_t a) {
    constexpr int RC = Plan<LEN, E>::RC;
    if constexpr (RC > 1 && SPAN % RC == 0) {
        if constexpr (RC % 2 == 1) {
            if constexpr (SPAN == RC) {
                return a;
            } else {
                return a + (a >> 4);
            }
        } else {
            constexpr int W = 128 / (int)sizeof(cx<T>);
            constexpr uint32_t D = (uint32_t)(RC / gcd_c(RC, W) * W);  // lcm(RC, W) >= 16: fits smem_elems
            return a + a / D;
        }
    } else {
        return a + (a >> 4);
    }
}
// Slot at a stage boundary: ridx for rows, sidx for interleaved columns.
template <typename T, int LEN, int COLS, int E, int SPAN>
__device__ __forceinline__ uint32_t bslot(uint32_t a, uint32_t col) {
    if constexpr (COLS == 1) {
        return ridx<T, LEN, E, SPAN>(a);
    } else {
        return sidx<COLS>(a, col);
    }
}

// Period of a boundary's slot map: every map above satisfies
//     slot(x + Q) = slot(x) + slot(Q)   for all x
// (Q = 16 / COLS for interleaved columns, 16 for a skewed row, D for a padded row,
// 1 for the plain index), and hence slot(x + c, col) = slot(x, col) + slot(c, 0)
// whenever x or c is a multiple of Q. Stage loops use that to compute one slot per
// butterfly group and reach the others by compile-time offsets.
template <typename T, int LEN, int COLS, int E, int SPAN>
constexpr int slot_period() {
    static_assert(COLS == 1 || 16 % COLS == 0, "interleaved columns must divide 16");
    if constexpr (COLS > 1) {
        return 16 / COLS;
    } else {
        constexpr int RC = Plan<LEN, E>::RC;
        if constexpr (RC > 1 && SPAN % RC == 0) {
            if constexpr (RC % 2 == 1) {
                return SPAN == RC ? 1 : 16;
            } else {
                constexpr int W = 128 / (int)sizeof(cx<T>);
                return RC / gcd_c(RC, W) * W;
            }
        } else {
            return 16;
        }
    }
}

// One Stockham stage of radix R at span P, from registers (already loaded
// with this stage's inputs) to shared memory. Thread tq handles the E/R
// butterfly groups i = tq + b*TC; group i reads elements i + r*LEN/R,
// multiplies by w_{R P}^{r k} (k = i mod P; w_{R P}^{j} = w_F^{j F/(R P)}),
// transforms, and writes element (i - k)*R + k + r*P.
template <typename T, int LEN, int COLS, int E, int R, int P, bool INV>
__device__ __forceinline__ void stage_to_smem(cx<T> *sm, cx<T> *v, uint32_t tq, uint32_t col, const TwTab<T> &tw) {
    constexpr int TC = LEN / E;
    constexpr int Q = slot_period<T, LEN, COLS, E, P * R>();
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        const uint32_t i = tq + (uint32_t)b * TC;
        const uint32_t k = i % P;
        if (P > 1) stage_twiddles<T, INV, R>(v + b * R, tw, k * (tw.F / (R * P)));
        dft<T, R, INV>(v + b * R);
        const uint32_t base = (i - k) * R + k;
        if constexpr (P % Q == 0 || (P == 1 && R % Q == 0)) {
            // offsets r*P are multiples of Q, or (P = 1, so k = 0) base = i*R is one
            const uint32_t s0 = bslot<T, LEN, COLS, E, P * R>(base, col);
#pragma unroll
            for (int r = 0; r < R; ++r) sm[s0 + bslot<T, LEN, COLS, E, P * R>((uint32_t)(r * P), 0)] = v[b * R + r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) sm[bslot<T, LEN, COLS, E, P * R>(base + (uint32_t)r * P, col)] = v[b * R + r];
        }
    }
}

// Load a stage's inputs from shared memory: group i = tq + b*TC, elements i + r*LEN/R
// (boundary of span SPAN, the reading stage's span).
template <typename T, int LEN, int COLS, int E, int R, int SPAN>
__device__ __forceinline__ void load_from_smem(const cx<T> *sm, cx<T> *v, uint32_t tq, uint32_t col) {
    constexpr int TC = LEN / E;
    constexpr int Q = slot_period<T, LEN, COLS, E, SPAN>();
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        const uint32_t i = tq + (uint32_t)b * TC;
        if constexpr ((LEN / R) % Q == 0) {  // offsets r*LEN/R are multiples of Q
            const uint32_t s0 = bslot<T, LEN, COLS, E, SPAN>(i, col);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = sm[s0 + bslot<T, LEN, COLS, E, SPAN>((uint32_t)(r * (LEN / R)), 0)];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = sm[bslot<T, LEN, COLS, E, SPAN>(i + (uint32_t)r * (LEN / R), col)];
        }
    }
}

// Last stage: twiddle + DFT in registers, results stay in registers.
template <typename T, int LEN, int COLS, int E, int R, int P, bool INV>
__device__ __forceinline__ void stage_in_regs(cx<T> *v, uint32_t tq, const TwTab<T> &tw) {
    constexpr int TC = LEN / E;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        const uint32_t i = tq + (uint32_t)b * TC;
        const uint32_t k = i % P;
        if (P > 1) stage_twiddles<T, INV, R>(v + b * R, tw, k * (tw.F / (R * P)));
        dft<T, R, INV>(v + b * R);
    }
}

// Power-of-two stages S .. q-1 of the forward transform (radix R0 first, then
// E), starting at span P0. Stage S's inputs are in registers when FROM_REGS,
// else in shared memory. The last stage leaves its outputs in registers.
template <typename T, int LEN, int COLS, int E, int S, int P0, bool FROM_REGS>
__device__ __forceinline__ void fwd_pow2(cx<T> *sm, cx<T> *v, uint32_t tq, uint32_t col, const TwTab<T> &tw) {
    using PL = Plan<LEN, E>;
    constexpr int R = (S == 0) ? PL::r0 : E;
    if constexpr (!FROM_REGS) {
        __syncthreads();
        load_from_smem<T, LEN, COLS, E, R, P0>(sm, v, tq, col);
    }
    if constexpr (S == PL::q - 1) {
        stage_in_regs<T, LEN, COLS, E, R, P0, false>(v, tq, tw);
    } else {
        if constexpr (!FROM_REGS) __syncthreads();
        stage_to_smem<T, LEN, COLS, E, R, P0, false>(sm, v, tq, col, tw);
        fwd_pow2<T, LEN, COLS, E, S + 1, P0 * R, false>(sm, v, tq, col, tw);
    }
}

// Power-of-two stages of the inverse transform: E, ..., E, R0 (stage S counts
// from the first). The first stage's inputs are in registers. With TO_SMEM the
// last stage writes its outputs to shared memory (an odd stage follows),
// otherwise they stay in registers.
// LAST is the index of the last power-of-two stage to run (q - 1, or q - 2 when
// the odd stage absorbs the radix-r0 stage).
template <typename T, int LEN, int COLS, int E, int S, int P0, bool TO_SMEM, int LAST = Plan<LEN, E>::q - 1>
__device__ __forceinline__ void inv_pow2(cx<T> *sm, cx<T> *v, uint32_t tq, uint32_t col, const TwTab<T> &tw) {
    using PL = Plan<LEN, E>;
    constexpr int R = (S == PL::q - 1) ? PL::r0 : E;
    if constexpr (S > 0) {
        __syncthreads();
        load_from_smem<T, LEN, COLS, E, R, P0>(sm, v, tq, col);
    }
    if constexpr (S == LAST && !TO_SMEM) {
        stage_in_regs<T, LEN, COLS, E, R, P0, true>(v, tq, tw);
    } else {
        if constexpr (S > 0) __syncthreads();
        stage_to_smem<T, LEN, COLS, E, R, P0, true>(sm, v, tq, col, tw);
        if constexpr (S < LAST) inv_pow2<T, LEN, COLS, E, S + 1, P0 * R, TO_SMEM, LAST>(sm, v, tq, col, tw);
    }
}

// Full power-of-two transform of length LEN on COLS interleaved columns. On
// entry v holds the first-stage inputs (forward: idx_r0 layout; inverse:
// idx_e layout); on exit v holds the outputs (forward: idx_e layout; inverse:
// idx_r0 layout). The caller must __syncthreads() before the call if shared
// memory is still being read from a previous transform.
template <typename T, int LEN, int COLS, int E, bool INV>
__device__ __forceinline__ void cta_fft(cx<T> *sm, cx<T> *v, uint32_t tq, uint32_t col, const TwTab<T> &tw) {
    static_assert(Plan<LEN, E>::RO == 1, "odd lengths use cta_fft_fwd_odd / cta_fft_inv_odd");
    if constexpr (!INV) {
        fwd_pow2<T, LEN, COLS, E, 0, 1, true>(sm, v, tq, col, tw);
    } else {
        inv_pow2<T, LEN, COLS, E, 0, 1, false>(sm, v, tq, col, tw);
    }
}

// Forward transform of a contiguous row of LEN = RO * 2^k elements (RO > 1).
// The first stage has the odd (or composite) radix RC = Plan::RC at span 1: group
// g = tq + j TC < LEN / RC reads elements g + r LEN / RC through ld(offset), the offset
// j TC + r LEN / RC counted from element tq (a compile-time constant, so the caller's
// base pointer for thread tq takes immediate offsets), transforms, and writes
// shared-memory slots g RC + r (odd_first_stage). The power-of-two stages follow
// (fwd_odd_rest); outputs end in registers (idx_e).
template <typename T, int LEN, int E, class Ld>
__device__ __forceinline__ void odd_first_stage(cx<T> *sm, uint32_t tq, Ld ld) {
    using PL = Plan<LEN, E>;
    constexpr int RC = PL::RC, K = LEN / RC, TC = PL::TC;
    constexpr int G = (K + TC - 1) / TC;  // groups per thread (the last may be partial)
#pragma unroll
    for (int j = 0; j < G; ++j) {
        const uint32_t g = tq + (uint32_t)j * TC;
        if (g < (uint32_t)K) {
            cx<T> u[RC];
#pragma unroll
            for (int r = 0; r < RC; ++r) u[r] = ld((uint32_t)(j * TC + r * K));
            dft_comp<T, PL::RO, PL::R0C, false>(u);
#pragma unroll
            for (int r = 0; r < RC; ++r) sm[ridx<T, LEN, E, RC>(g * RC + (uint32_t)r)] = u[r];
        }
    }
}

template <typename T, int LEN, int E>
__device__ __forceinline__ void fwd_odd_rest(cx<T> *sm, cx<T> *v, uint32_t tq, const TwTab<T> &tw) {
    using PL = Plan<LEN, E>;
    fwd_pow2<T, LEN, 1, E, PL::FOLD ? 1 : 0, PL::RC, false>(sm, v, tq, 0, tw);
}

template <typename T, int LEN, int E, class Ld>
__device__ __forceinline__ void cta_fft_fwd_odd(cx<T> *sm, cx<T> *v, uint32_t tq, const TwTab<T> &tw, Ld ld) {
    odd_first_stage<T, LEN, E>(sm, tq, ld);
    fwd_odd_rest<T, LEN, E>(sm, v, tq, tw);
}

// Inverse transform of a row (RO > 1): power-of-two stages from registers
// (idx_e layout) into shared memory, then the odd (or composite) last stage at
// span K = LEN / RC: group g = tq + j TC < K reads slots g + r K, takes the twiddles
// w_LEN^{-r g}, transforms, and its output g + r K goes through st(j TC + r K, value)
// (offset from element tq, as for ld above).
template <typename T, int LEN, int E, class St>
__device__ __forceinline__ void cta_fft_inv_odd(cx<T> *sm, cx<T> *v, uint32_t tq, const TwTab<T> &tw, St st) {
    using PL = Plan<LEN, E>;
    constexpr int RC = PL::RC, K = LEN / RC, TC = PL::TC;
    constexpr int G = (K + TC - 1) / TC;
    inv_pow2<T, LEN, 1, E, 0, 1, true, PL::FOLD ? PL::q - 2 : PL::q - 1>(sm, v, tq, 0, tw);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < G; ++j) {
        const uint32_t g = tq + (uint32_t)j * TC;
        if (g < (uint32_t)K) {
            cx<T> u[RC];
            if constexpr (K % slot_period<T, LEN, 1, E, K>() == 0) {  // offsets r*K are multiples of the period
                const uint32_t s0 = ridx<T, LEN, E, K>(g);
#pragma unroll
                for (int r = 0; r < RC; ++r) u[r] = sm[s0 + ridx<T, LEN, E, K>((uint32_t)(r * K))];
            } else {
#pragma unroll
                for (int r = 0; r < RC; ++r) u[r] = sm[ridx<T, LEN, E, K>(g + (uint32_t)r * K)];
            }
            stage_twiddles<T, true, RC>(u, tw, g * (tw.F / LEN));
            dft_comp<T, PL::RO, PL::R0C, true>(u);
#pragma unroll
            for (int r = 0; r < RC; ++r) st((uint32_t)(j * TC + r * K), u[r]);
        }
    }
}

}  // namespace pa

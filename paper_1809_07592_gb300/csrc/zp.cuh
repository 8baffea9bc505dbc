// zp.cuh -- arithmetic modulo the prime p = 2^64 - 2^32 + 1 for the exact
// number-theoretic transform (paper Section 1 names the fast number-theoretic
// transform as the exact alternative to the FFT for Toeplitz hashing).
//
// p - 1 = 2^32 * 3 * 5 * 17 * 257 * 65537, so power-of-two transform lengths up
// to 2^32 have roots of unity. 2^96 = -1 (mod p), so 2 has order 192 and
// 2^6 is a primitive 32nd root of unity: the in-register DFTs use powers of
// 2^6, and the host picks the length-L root w_L with w_L^(L/32) = 2^6 so that
// the table twiddles and the in-register roots belong to one root system.
//
// Residues are kept canonical, in [0, p), after every operation.
#pragma once

#include <cstdint>

namespace pa {

struct Zp {};  // tag type selecting modular arithmetic

constexpr uint64_t kP = 0xFFFFFFFF00000001ull;  // 2^64 - 2^32 + 1
constexpr uint64_t kEps = 0xFFFFFFFFull;        // 2^64 mod p = 2^32 - 1

__host__ __device__ __forceinline__ uint64_t zp_add(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    // a + b < 2p; on a carry out of 64 bits the true sum is s + 2^64, and
    // s + 2^64 - p = s - p (mod 2^64)
    if (s < a || s >= kP) s -= kP;
    return s;
}

__host__ __device__ __forceinline__ uint64_t zp_sub(uint64_t a, uint64_t b) {
    uint64_t d = a - b;
    if (a < b) d += kP;
    return d;
}

// Reduce hi * 2^64 + lo. With hi = hh * 2^32 + hl: 2^64 = 2^32 - 1 and
// 2^96 = -1 (mod p), so the value is lo + hl * (2^32 - 1) - hh (mod p).
__host__ __device__ __forceinline__ uint64_t zp_reduce(uint64_t hi, uint64_t lo) {
    const uint64_t hh = hi >> 32, hl = hi & 0xFFFFFFFFull;
    uint64_t t = lo - hh;
    if (lo < hh) t -= kEps;  // borrow: -2^64 = -(2^32 - 1)
    const uint64_t u = hl * kEps;  // < 2^64
    uint64_t r = t + u;
    if (r < u) r += kEps;  // carry: 2^64 = 2^32 - 1
    if (r >= kP) r -= kP;
    return r;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint64_t zp_mul(uint64_t a, uint64_t b) { return zp_reduce(__umul64hi(a, b), a * b); }
#endif

// 2^k mod p for 0 <= k < 192 (host and device constexpr).
__host__ __device__ constexpr uint64_t zp_pow2(int k) {
    // 2^k for k < 64 is itself (< p); 2^(64+j) = (2^32 - 1) 2^j for j < 32
    // (< p); 2^(96+j) = -2^j for j < 96.
    return k < 64 ? (1ull << k)
           : k < 96 ? (kEps << (k - 64))
           : k < 160 ? (kP - (1ull << (k - 96)))
                     : (kP - (kEps << (k - 160)));
}

template <> struct Arith<Zp> {
    using E = unsigned long long;
    static __device__ __forceinline__ E add(E a, E b) { return zp_add(a, b); }
    static __device__ __forceinline__ E sub(E a, E b) { return zp_sub(a, b); }
    static __device__ __forceinline__ E mul(E a, E b) { return zp_mul(a, b); }
    // x * w32^j (forward) or x * w32^-j (inverse) with w32 = 2^6.
    template <bool INV> static __device__ __forceinline__ E rot32(E x, int j) {
        if (j == 0) return x;
        const int k = INV ? (192 - 6 * j) : 6 * j;
        return zp_mul(x, zp_pow2(k));
    }
    // w_F^e (forward) or w_F^-e = w_F^(F-e) (inverse) from the stage table.
    template <bool INV> static __device__ __forceinline__ E fine(const TwTab<Zp> &t, uint32_t e) {
        if (INV && e) e = t.F - e;
        return __ldg(t.fine + e);
    }
    // w_L^e (forward) or w_L^-e = w_L^(L-e) (inverse) from the two-level table.
    template <bool INV> static __device__ __forceinline__ E omega(const TwTab<Zp> &t, uint32_t e) {
        if (INV) e = (uint32_t)((0u - e) & ((1u << t.lgL) - 1u));
        const E a = __ldg(t.hi + (e >> t.B));
        const E b = __ldg(t.lo + (e & ((1u << t.B) - 1u)));
        return zp_mul(a, b);
    }
};

}  // namespace pa

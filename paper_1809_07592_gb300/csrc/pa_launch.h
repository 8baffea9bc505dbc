// pa_launch.h -- host-side launchers of the pass kernels (declarations).
//
// Each launcher picks the kernel instance for its pass length, sets its dynamic
// shared memory and launches it on the given stream. Strided passes have
// power-of-two lengths 2^lgLEN; innermost passes have lengths RO * 2^lg with an
// odd factor RO in {1, 3, 5, 9} (smooth transform lengths). The definitions live
// in pa_launch.cuh, instantiated per arithmetic type (pa_f32.cu, pa_f64.cu,
// pa_zp.cu) and, for the odd innermost lengths, per (type, RO) (pa_*_r*.cu).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "fft_core.cuh"

namespace pa {

// Per-type kernel shape: E complex values per thread, COLS columns per CTA in
// the strided passes. FP64 halves both to keep registers and shared memory
// within one SM's budget.
template <typename T> struct Shape;
template <> struct Shape<float> { static constexpr int E = 16, COLS = 16; };
template <> struct Shape<double> { static constexpr int E = 8, COLS = 8; };
template <> struct Shape<Zp> { static constexpr int E = 8, COLS = 8; };
// Columns per CTA of a strided pass of length LEN: single precision takes 8 instead of 16 at
// LEN = 1024 (512 threads, two CTAs per SM instead of one).
template <typename T, int LEN>
constexpr int strided_cols() {
    return (std::is_same<T, float>::value && LEN >= 1024) ? 8 : Shape<T>::COLS;
}

// Supported pass lengths (log2).
constexpr int kMinLgStrided = 6, kMaxLgStrided = 10;
template <typename T> struct MaxLgMiddle;
template <> struct MaxLgMiddle<float> { static constexpr int v = 14; };
template <> struct MaxLgMiddle<double> { static constexpr int v = 13; };
template <> struct MaxLgMiddle<Zp> { static constexpr int v = 13; };
constexpr int kMinLgMiddle = 6;

// Zero the per-key popcounts and margins of a batch (the level-1 forward pass accumulates the popcounts).
cudaError_t launch_zero_keys(uint32_t nkeys, uint32_t *popc, uint32_t *margin_bits, cudaStream_t st);

// Round x[0 .. count) in place to `bits` explicit significand bits (1 <= bits <= 22; other
// values leave x as it is): the storage-precision study of pa_plan_set_storage_bits.
cudaError_t launch_round_significand(float *x, uint64_t count, uint32_t bits, cudaStream_t st);

// Level-1 forward pass of key pairs; also adds each key's popcount into popc[k]
// (which must be zero beforehand: launch_zero_keys). The transform input is key
// bits koff .. koff+n-1 (koff = m for the modified Toeplitz hash).
// pack: one key per slot in a half-length transform (element t = key bits 2t, 2t+1).
template <typename T>
cudaError_t launch_fwd_keys(int lgLEN, const uint64_t *keys, uint32_t nkeys, uint64_t kstride, uint64_t n,
                            cx<T> *W, uint64_t L, uint32_t pairs, TwTab<T> tw, uint32_t *popc, cudaStream_t st,
                            uint64_t koff = 0, bool pack = false);
// pack: the seed of a length-2L convolution in a length-L transform (positions 2t, 2t+1).
template <typename T>
cudaError_t launch_fwd_seed(int lgLEN, const uint64_t *seed, uint64_t n, uint64_t m, cx<T> *W, uint64_t L,
                            TwTab<T> tw, cudaStream_t st, bool pack = false);
// S: innermost length (the stride of the middle strided pass).
template <typename T>
cudaError_t launch_mid(int lgLEN, bool inverse, cx<T> *W, uint64_t L, uint32_t S, uint32_t pairs, TwTab<T> tw,
                       cudaStream_t st);
// Innermost pass of length ro * 2^lg. mode 0: the fused convolution step; mode 1:
// the seed spectrum.
template <typename T>
cudaError_t launch_middle(int ro, int lg, int mode, cx<T> *W, cx<T> *spec, uint64_t L, uint32_t pairs, TwTab<T> tw,
                          cx<T> scale, cudaStream_t st);
template <typename T, int RO>
cudaError_t launch_middle_odd(int lg, int mode, cx<T> *W, cx<T> *spec, uint64_t L, uint32_t pairs, TwTab<T> tw,
                              cx<T> scale, cudaStream_t st);

// Limits of the odd innermost lengths RO * 2^lg: a CTA has RO * 2^lg / E threads
// (at most 1024, or 512 per row for the two-row split kernel).
constexpr int kMinLgOdd = 7, kMaxLgOdd = 11;
template <typename T>
constexpr bool odd_inner_ok(int ro, int lg, bool split) {
    return lg >= kMinLgOdd && lg <= kMaxLgOdd && (long long)ro * (1ll << lg) / Shape<T>::E <= (split ? 512 : 1024);
}
// Level-1 inverse pass with the bit output. With xkeys, output bit i of key k is
// XORed with bit i of xkeys + k*xstride (the identity block of the modified hash).
// With ctl != nullptr (three device words, zero before the first launch: error bits,
// tile ticket, CTAs done), FP32 pairs with pass lengths up to 256 run the persistent
// TMA-staged kernel; a copy wait there that runs out of time sets bit 0 of ctl[0].
// expire_ns != 0 (test hook) makes that kernel copy nothing and let its wait run out.
template <typename T>
cudaError_t launch_inv_bits(int lgLEN, const cx<T> *W, uint64_t L, uint64_t m, uint32_t nkeys,
                            const uint32_t *popc, uint32_t *margin_bits, uint64_t *out, uint64_t ostride,
                            uint32_t pairs, TwTab<T> tw, cudaStream_t st, const uint64_t *xkeys = nullptr,
                            uint64_t xstride = 0, bool pack = false, uint32_t *ctl = nullptr,
                            uint32_t expire_ns = 0);
// Whether launch_inv_bits runs the TMA-staged kernel for this type and pass length.
constexpr bool inv_bits_staged(uint64_t elem_bytes, int lgLEN) { return elem_bytes == 8 && lgLEN <= 8; }

// Tiled-copy descriptor of a row-major array of rows x cols 8-byte elements at base, copied
// in boxes of box_cols x box_rows (the cuTensorMapEncodeTiled encoder, resolved from the
// driver at run time). false if the driver offers no encoder or rejects the layout.
bool encode_tile_map(CUtensorMap *map, const void *base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                     uint32_t box_rows);

// ---- uneven batch (complex arithmetic only: the Eq. 5-10 split needs conjugation) ----
struct BlockDev;
template <typename T> struct MaxLgSplit;
template <> struct MaxLgSplit<float> { static constexpr int v = 13; };
template <> struct MaxLgSplit<double> { static constexpr int v = 12; };

// Zero popc[id] and margin_bits[id] of every block (launch_fwd_keyseed accumulates the popcounts).
cudaError_t launch_zero_blocks(const BlockDev *blocks, uint32_t nblocks, uint32_t *popc, uint32_t *margin_bits,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_fwd_keyseed(int lgLEN, const BlockDev *blocks, uint32_t nblocks, cx<T> *W, uint64_t L,
                               TwTab<T> tw, uint32_t *popc, cudaStream_t st);
template <typename T>
cudaError_t launch_middle_split(int ro, int lg, const cx<T> *Wf, cx<T> *Wi, uint64_t L, uint32_t nblocks,
                                uint32_t lgL1, uint32_t lgM, TwTab<T> tw, cudaStream_t st);
template <typename T, int RO>
cudaError_t launch_middle_split_odd(int lg, const cx<T> *Wf, cx<T> *Wi, uint64_t L, uint32_t nblocks, uint32_t lgL1,
                                    uint32_t lgM, TwTab<T> tw, cudaStream_t st);
template <typename T>
cudaError_t launch_inv_bits_blocks(int lgLEN, const cx<T> *Wi, uint64_t L, const BlockDev *blocks, uint32_t nblocks,
                                   const uint32_t *popc, uint32_t *margin_bits, TwTab<T> tw, cudaStream_t st);

// ---- single keys in half-length transforms (complex arithmetic only) ----
// Innermost pass of length ro * 2^lg over a length-N slot (slots of N elements from W):
// mode 0 multiplies with the seed tables (3N values: E_s, O_s, w_N^k O_s, times 1/N) and
// transforms back; mode 1 builds those tables from the packed seed's transform (scale 1/N).
template <typename T>
cudaError_t launch_middle_real(int ro, int lg, int mode, cx<T> *W, cx<T> *tabs, uint64_t N, uint32_t lgL1,
                               uint32_t lgM, TwTab<T> tw, T scale, uint32_t slots, cudaStream_t st);
template <typename T, int RO>
cudaError_t launch_middle_real_odd(int lg, int mode, cx<T> *W, cx<T> *tabs, uint64_t N, uint32_t lgL1, uint32_t lgM,
                                   TwTab<T> tw, T scale, uint32_t slots, cudaStream_t st);

}  // namespace pa

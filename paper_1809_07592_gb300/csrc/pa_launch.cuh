// pa_launch.cuh -- launcher definitions; included by the per-type .cu files.
#pragma once

#include <type_traits>

#include "pa_kernels.cuh"
#include "pa_launch.h"

namespace pa {

// Opt a kernel into more than 48 KB of dynamic shared memory, once per kernel
// and device: later launches (and launches inside a stream capture) make no
// attribute call.
bool smem_configured(const void *kernel, int device);
void smem_mark_configured(const void *kernel, int device);

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    const void *key = reinterpret_cast<const void *>(kernel);
    if (smem_configured(key, dev)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) smem_mark_configured(key, dev);
    return e;
}

template <typename T, int LEN, int COLS>
constexpr size_t smem_bytes() {
    return (size_t)smem_elems<LEN, COLS>() * sizeof(cx<T>);
}

// Calls f(std::integral_constant<int, LEN>) for LEN = 2^lg in [2^LO, 2^HI].
template <int LO, int HI, typename F>
static cudaError_t by_len(int lg, F &&f) {
    if constexpr (LO > HI) {
        return cudaErrorInvalidValue;
    } else {
        if (lg == LO) return f(std::integral_constant<int, (1 << LO)>{});
        return by_len<LO + 1, HI>(lg, f);
    }
}

template <typename T, int LEN, bool PACK>
cudaError_t fwd_keys_at(const uint64_t *keys, uint32_t nkeys, uint64_t kstride, uint64_t n, cx<T> *W, uint64_t L,
                        uint32_t pairs, TwTab<T> tw, uint32_t *popc, cudaStream_t st, uint64_t koff) {
    constexpr int E = Shape<T>::E, COLS = strided_cols<T, LEN>();
    auto kern = k_fwd_keys<T, LEN, COLS, E, PACK>;
    constexpr size_t sb = smem_bytes<T, LEN, COLS>() + stage_bytes<T, LEN, COLS>();
    cudaError_t e = set_smem(kern, sb);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((L / LEN) / COLS), pairs);
    kern<<<grid, COLS * LEN / E, sb, st>>>(keys, nkeys, kstride, n, W, L, tw, popc, koff);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fwd_keys(int lgLEN, const uint64_t *keys, uint32_t nkeys, uint64_t kstride, uint64_t n,
                            cx<T> *W, uint64_t L, uint32_t pairs, TwTab<T> tw, uint32_t *popc, cudaStream_t st,
                            uint64_t koff, bool pack) {
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        if constexpr (!std::is_same<T, Zp>::value) {
            if (pack) return fwd_keys_at<T, LEN, true>(keys, nkeys, kstride, n, W, L, pairs, tw, popc, st, koff);
        } else {
            if (pack) return cudaErrorInvalidValue;  // the exact transform has no half-length packing
        }
        return fwd_keys_at<T, LEN, false>(keys, nkeys, kstride, n, W, L, pairs, tw, popc, st, koff);
    });
}

template <typename T, int LEN, bool PACK>
cudaError_t fwd_seed_at(const uint64_t *seed, uint64_t n, uint64_t m, cx<T> *W, uint64_t L, TwTab<T> tw,
                        cudaStream_t st) {
    constexpr int E = Shape<T>::E, COLS = strided_cols<T, LEN>();
    auto kern = k_fwd_seed<T, LEN, COLS, E, PACK>;
    constexpr size_t sb = smem_bytes<T, LEN, COLS>();
    cudaError_t e = set_smem(kern, sb);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((L / LEN) / COLS), 1);
    kern<<<grid, COLS * LEN / E, sb, st>>>(seed, n, m, W, L, tw);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fwd_seed(int lgLEN, const uint64_t *seed, uint64_t n, uint64_t m, cx<T> *W, uint64_t L,
                            TwTab<T> tw, cudaStream_t st, bool pack) {
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        if constexpr (!std::is_same<T, Zp>::value) {
            if (pack) return fwd_seed_at<T, LEN, true>(seed, n, m, W, L, tw, st);
        } else {
            if (pack) return cudaErrorInvalidValue;
        }
        return fwd_seed_at<T, LEN, false>(seed, n, m, W, L, tw, st);
    });
}

template <typename T>
cudaError_t launch_mid(int lgLEN, bool inverse, cx<T> *W, uint64_t L, uint32_t S, uint32_t pairs, TwTab<T> tw,
                       cudaStream_t st) {
    constexpr int E = Shape<T>::E;
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        constexpr int COLS = strided_cols<T, LEN>();
        constexpr size_t sb = smem_bytes<T, LEN, COLS>();
        const uint64_t nblk = L / ((uint64_t)LEN * S);
        const uint32_t mult = (uint32_t)(L / ((uint64_t)LEN * S));
        dim3 grid((unsigned)(S / COLS), (unsigned)(nblk * pairs));
        if (inverse) {
            auto kern = k_mid<T, LEN, COLS, E, true>;
            cudaError_t e = set_smem(kern, sb);
            if (e != cudaSuccess) return e;
            kern<<<grid, COLS * LEN / E, sb, st>>>(W, L, S, mult, tw);
        } else {
            auto kern = k_mid<T, LEN, COLS, E, false>;
            cudaError_t e = set_smem(kern, sb);
            if (e != cudaSuccess) return e;
            kern<<<grid, COLS * LEN / E, sb, st>>>(W, L, S, mult, tw);
        }
        return cudaGetLastError();
    });
}

// Persistent grid of a kernel: resident CTAs per SM (occupancy query) times the SM
// count. `cache` (one per kernel instance) keeps the product per device.
template <typename K>
cudaError_t persistent_ctas(K kern, int threads, size_t smem, int *cache, uint32_t *ctas) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
    if (cache[dev] == 0) {
        int o = 0, n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, threads, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (o < 1) o = 1;
        cache[dev] = o * n;
    }
    *ctas = (uint32_t)cache[dev];
    return cudaSuccess;
}

template <typename T, int LEN>
cudaError_t middle_at(int mode, cx<T> *W, cx<T> *spec, uint64_t L, uint32_t pairs, TwTab<T> tw, cx<T> scale,
                      cudaStream_t st) {
    constexpr int E = Shape<T>::E;
    constexpr size_t sb = smem_bytes<T, LEN, 1>();
    dim3 grid((unsigned)(L / LEN), pairs);
    if (mode == 0) {
        auto kern = k_middle<T, LEN, E, 0>;
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        kern<<<grid, LEN / E, sb, st>>>(W, spec, L, tw, scale);
    } else {
        auto kern = k_middle<T, LEN, E, 1>;
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        kern<<<grid, LEN / E, sb, st>>>(W, spec, L, tw, scale);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_middle(int ro, int lg, int mode, cx<T> *W, cx<T> *spec, uint64_t L, uint32_t pairs, TwTab<T> tw,
                          cx<T> scale, cudaStream_t st) {
    if (ro == 1) {
        return by_len<kMinLgMiddle, MaxLgMiddle<T>::v>(lg, [&](auto c) {
            return middle_at<T, decltype(c)::value>(mode, W, spec, L, pairs, tw, scale, st);
        });
    }
    if constexpr (std::is_same<T, Zp>::value) {
        return cudaErrorInvalidValue;  // the exact transform keeps power-of-two lengths
    } else {
        if (ro == 3) return launch_middle_odd<T, 3>(lg, mode, W, spec, L, pairs, tw, scale, st);
        if (ro == 5) return launch_middle_odd<T, 5>(lg, mode, W, spec, L, pairs, tw, scale, st);
        if (ro == 9) return launch_middle_odd<T, 9>(lg, mode, W, spec, L, pairs, tw, scale, st);
        return cudaErrorInvalidValue;
    }
}

// Odd innermost lengths RO * 2^lg, lg in [kMinLgOdd, kMaxLgOdd], where the CTA fits.
template <typename T, int RO, int LG = kMinLgOdd>
cudaError_t odd_middle_dispatch(int lg, int mode, cx<T> *W, cx<T> *spec, uint64_t L, uint32_t pairs, TwTab<T> tw,
                                cx<T> scale, cudaStream_t st) {
    if constexpr (LG > kMaxLgOdd) {
        return cudaErrorInvalidValue;
    } else {
        if (lg == LG) {
            if constexpr (odd_inner_ok<T>(RO, LG, false)) {
                return middle_at<T, RO * (1 << LG)>(mode, W, spec, L, pairs, tw, scale, st);
            } else {
                return cudaErrorInvalidValue;
            }
        }
        return odd_middle_dispatch<T, RO, LG + 1>(lg, mode, W, spec, L, pairs, tw, scale, st);
    }
}

template <typename T, int RO>
cudaError_t launch_middle_odd(int lg, int mode, cx<T> *W, cx<T> *spec, uint64_t L, uint32_t pairs, TwTab<T> tw,
                              cx<T> scale, cudaStream_t st) {
    return odd_middle_dispatch<T, RO>(lg, mode, W, spec, L, pairs, tw, scale, st);
}

// The TMA-staged persistent form of the level-1 inverse pass (k_inv_bits_tma): FP32 pair
// form, LEN <= 256 (one tiled copy per tile), when the driver offers the tensor-map encoder.
template <int LEN>
cudaError_t inv_bits_tma_at(const float2 *W, uint64_t L, uint64_t m, uint32_t nkeys, const uint32_t *popc,
                            uint32_t *margin_bits, uint64_t *out, uint64_t ostride, uint32_t pairs, TwTab<float> tw,
                            cudaStream_t st, const uint64_t *xkeys, uint64_t xstride, uint32_t *ctl,
                            uint32_t expire_ns, bool *done) {
    *done = false;
    constexpr int COLS = Shape<float>::COLS;
    const uint64_t S = L / LEN;
    CUtensorMap map;
    if (!encode_tile_map(&map, W, S, (uint64_t)pairs * LEN, COLS, LEN)) return cudaSuccess;  // no encoder: plain kernel
    auto kern = k_inv_bits_tma<LEN>;
    // staged tile + exchange buffer + 128 bytes to align the tile for the tiled copy
    constexpr size_t sb = (size_t)LEN * COLS * sizeof(float2) + smem_bytes<float, LEN, COLS>() + 128;
    cudaError_t e = set_smem(kern, sb);
    if (e != cudaSuccess) return e;
    static int cache[16] = {0};  // resident CTAs on each device
    uint32_t ctas = 0;
    e = persistent_ctas(kern, LEN, sb, cache, &ctas);
    if (e != cudaSuccess) return e;
    const uint64_t ntiles = (S / COLS) * pairs;
    if (ntiles > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    const uint32_t grid = (uint32_t)(ntiles < ctas ? ntiles : ctas);
    kern<<<grid, LEN, sb, st>>>(map, L, m, nkeys, pairs, popc, margin_bits, out, ostride, tw, xkeys, xstride, ctl,
                                expire_ns);
    *done = true;
    return cudaGetLastError();
}

template <typename T, int LEN, bool PACK>
cudaError_t inv_bits_at(const cx<T> *W, uint64_t L, uint64_t m, uint32_t nkeys, const uint32_t *popc,
                        uint32_t *margin_bits, uint64_t *out, uint64_t ostride, uint32_t pairs, TwTab<T> tw,
                        cudaStream_t st, const uint64_t *xkeys, uint64_t xstride, uint32_t *ctl,
                        uint32_t expire_ns) {
    constexpr int E = Shape<T>::E, COLS = strided_cols<T, LEN>();
    if constexpr (std::is_same<T, float>::value && !PACK && LEN <= 256) {
        if (ctl != nullptr) {
            bool done = false;
            cudaError_t e = inv_bits_tma_at<LEN>(W, L, m, nkeys, popc, margin_bits, out, ostride, pairs, tw, st, xkeys,
                                                 xstride, ctl, expire_ns, &done);
            if (e != cudaSuccess || done) return e;
        }
    }
    auto kern = k_inv_bits<T, LEN, COLS, E, PACK>;
    constexpr size_t sb = smem_bytes<T, LEN, COLS>();
    cudaError_t e = set_smem(kern, sb);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((L / LEN) / COLS), pairs);
    kern<<<grid, COLS * LEN / E, sb, st>>>(W, L, m, nkeys, popc, margin_bits, out, ostride, tw, xkeys, xstride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inv_bits(int lgLEN, const cx<T> *W, uint64_t L, uint64_t m, uint32_t nkeys,
                            const uint32_t *popc, uint32_t *margin_bits, uint64_t *out, uint64_t ostride,
                            uint32_t pairs, TwTab<T> tw, cudaStream_t st, const uint64_t *xkeys,
                            uint64_t xstride, bool pack, uint32_t *ctl, uint32_t expire_ns) {
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        if constexpr (!std::is_same<T, Zp>::value) {
            if (pack)
                return inv_bits_at<T, LEN, true>(W, L, m, nkeys, popc, margin_bits, out, ostride, pairs, tw, st,
                                                 xkeys, xstride, nullptr, 0u);
        } else {
            if (pack) return cudaErrorInvalidValue;
        }
        return inv_bits_at<T, LEN, false>(W, L, m, nkeys, popc, margin_bits, out, ostride, pairs, tw, st, xkeys,
                                          xstride, ctl, expire_ns);
    });
}

#define PA_INSTANTIATE_LAUNCHERS(T)                                                                              \
    template cudaError_t launch_fwd_keys<T>(int, const uint64_t *, uint32_t, uint64_t, uint64_t, cx<T> *,        \
                                            uint64_t, uint32_t, TwTab<T>, uint32_t *, cudaStream_t, uint64_t,    \
                                            bool);                                                               \
    template cudaError_t launch_fwd_seed<T>(int, const uint64_t *, uint64_t, uint64_t, cx<T> *, uint64_t,        \
                                            TwTab<T>, cudaStream_t, bool);                                       \
    template cudaError_t launch_mid<T>(int, bool, cx<T> *, uint64_t, uint32_t, uint32_t, TwTab<T>,               \
                                       cudaStream_t);                                                           \
    template cudaError_t launch_middle<T>(int, int, int, cx<T> *, cx<T> *, uint64_t, uint32_t, TwTab<T>, cx<T>,  \
                                          cudaStream_t);                                                        \
    template cudaError_t launch_inv_bits<T>(int, const cx<T> *, uint64_t, uint64_t, uint32_t, const uint32_t *,  \
                                            uint32_t *, uint64_t *, uint64_t, uint32_t, TwTab<T>, cudaStream_t,  \
                                            const uint64_t *, uint64_t, bool, uint32_t *, uint32_t);

template <typename T>
cudaError_t launch_fwd_keyseed(int lgLEN, const BlockDev *blocks, uint32_t nblocks, cx<T> *W, uint64_t L,
                               TwTab<T> tw, uint32_t *popc, cudaStream_t st) {
    constexpr int E = Shape<T>::E;
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        constexpr int COLS = strided_cols<T, LEN>();
        auto kern = k_fwd_keyseed<T, LEN, COLS, E>;
        constexpr size_t sb = smem_bytes<T, LEN, COLS>() + 2 * stage_bytes<T, LEN, COLS>();  // 64-bit stage
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((L / LEN) / COLS), nblocks);
        kern<<<grid, COLS * LEN / E, sb, st>>>(blocks, W, L, tw, popc);
        return cudaGetLastError();
    });
}

template <typename T, int LEN>
cudaError_t split_at(const cx<T> *Wf, cx<T> *Wi, uint64_t L, uint32_t nblocks, uint32_t lgL1, uint32_t lgM,
                     TwTab<T> tw, cudaStream_t st) {
    constexpr int E = Shape<T>::E;
    auto kern = k_middle_split<T, LEN, E>;
    constexpr size_t sb = 2 * smem_bytes<T, LEN, 1>();
    cudaError_t e = set_smem(kern, sb);
    if (e != cudaSuccess) return e;
    const uint32_t R = (uint32_t)(L / LEN);
    dim3 grid(R / 2 + 1, (nblocks + 1) / 2);
    kern<<<grid, 2 * (LEN / E), sb, st>>>(Wf, Wi, L, nblocks, lgL1, lgM, tw, (T)(1.0 / (double)L));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_middle_split(int ro, int lg, const cx<T> *Wf, cx<T> *Wi, uint64_t L, uint32_t nblocks,
                                uint32_t lgL1, uint32_t lgM, TwTab<T> tw, cudaStream_t st) {
    if (ro == 1) {
        return by_len<kMinLgMiddle, MaxLgSplit<T>::v>(lg, [&](auto c) {
            return split_at<T, decltype(c)::value>(Wf, Wi, L, nblocks, lgL1, lgM, tw, st);
        });
    }
    if (ro == 3) return launch_middle_split_odd<T, 3>(lg, Wf, Wi, L, nblocks, lgL1, lgM, tw, st);
    if (ro == 5) return launch_middle_split_odd<T, 5>(lg, Wf, Wi, L, nblocks, lgL1, lgM, tw, st);
    if (ro == 9) return launch_middle_split_odd<T, 9>(lg, Wf, Wi, L, nblocks, lgL1, lgM, tw, st);
    return cudaErrorInvalidValue;
}

template <typename T, int RO, int LG = kMinLgOdd>
cudaError_t odd_split_dispatch(int lg, const cx<T> *Wf, cx<T> *Wi, uint64_t L, uint32_t nblocks, uint32_t lgL1,
                               uint32_t lgM, TwTab<T> tw, cudaStream_t st) {
    if constexpr (LG > kMaxLgOdd) {
        return cudaErrorInvalidValue;
    } else {
        if (lg == LG) {
            if constexpr (odd_inner_ok<T>(RO, LG, true)) {
                return split_at<T, RO * (1 << LG)>(Wf, Wi, L, nblocks, lgL1, lgM, tw, st);
            } else {
                return cudaErrorInvalidValue;
            }
        }
        return odd_split_dispatch<T, RO, LG + 1>(lg, Wf, Wi, L, nblocks, lgL1, lgM, tw, st);
    }
}

template <typename T, int RO>
cudaError_t launch_middle_split_odd(int lg, const cx<T> *Wf, cx<T> *Wi, uint64_t L, uint32_t nblocks, uint32_t lgL1,
                                    uint32_t lgM, TwTab<T> tw, cudaStream_t st) {
    return odd_split_dispatch<T, RO>(lg, Wf, Wi, L, nblocks, lgL1, lgM, tw, st);
}

template <typename T>
cudaError_t launch_inv_bits_blocks(int lgLEN, const cx<T> *Wi, uint64_t L, const BlockDev *blocks, uint32_t nblocks,
                                   const uint32_t *popc, uint32_t *margin_bits, TwTab<T> tw, cudaStream_t st) {
    constexpr int E = Shape<T>::E;
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        constexpr int COLS = strided_cols<T, LEN>();
        auto kern = k_inv_bits_blocks<T, LEN, COLS, E>;
        constexpr size_t sb = smem_bytes<T, LEN, COLS>();
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((L / LEN) / COLS), (nblocks + 1) / 2);
        kern<<<grid, COLS * LEN / E, sb, st>>>(Wi, L, blocks, nblocks, popc, margin_bits, tw);
        return cudaGetLastError();
    });
}

#define PA_INSTANTIATE_UNEVEN(T)                                                                                 \
    template cudaError_t launch_fwd_keyseed<T>(int, const BlockDev *, uint32_t, cx<T> *, uint64_t, TwTab<T>,     \
                                               uint32_t *, cudaStream_t);                                       \
    template cudaError_t launch_middle_split<T>(int, int, const cx<T> *, cx<T> *, uint64_t, uint32_t, uint32_t,  \
                                                uint32_t, TwTab<T>, cudaStream_t);                               \
    template cudaError_t launch_inv_bits_blocks<T>(int, const cx<T> *, uint64_t, const BlockDev *, uint32_t,     \
                                                   const uint32_t *, uint32_t *, TwTab<T>, cudaStream_t);        \
    template cudaError_t launch_middle_real<T>(int, int, int, cx<T> *, cx<T> *, uint64_t, uint32_t, uint32_t,    \
                                               TwTab<T>, T, uint32_t, cudaStream_t);

// Single-key half-length innermost pass (k_middle_real): same lengths as the split pass.
template <typename T, int LEN>
cudaError_t real_at(int mode, cx<T> *W, cx<T> *tabs, uint64_t N, uint32_t lgL1, uint32_t lgM, TwTab<T> tw, T scale,
                    uint32_t slots, cudaStream_t st) {
    constexpr int E = Shape<T>::E;
    constexpr size_t sb = 2 * smem_bytes<T, LEN, 1>();
    const uint32_t R = (uint32_t)(N / LEN);
    dim3 grid(R / 2 + 1, slots);
    if (mode == 0) {
        auto kern = k_middle_real<T, LEN, E, 0>;
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        kern<<<grid, 2 * (LEN / E), sb, st>>>(W, tabs, N, lgL1, lgM, tw, scale);
    } else {
        auto kern = k_middle_real<T, LEN, E, 1>;
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        kern<<<grid, 2 * (LEN / E), sb, st>>>(W, tabs, N, lgL1, lgM, tw, scale);
    }
    return cudaGetLastError();
}

template <typename T, int RO, int LG = kMinLgOdd>
cudaError_t real_odd_dispatch(int lg, int mode, cx<T> *W, cx<T> *tabs, uint64_t N, uint32_t lgL1, uint32_t lgM,
                              TwTab<T> tw, T scale, uint32_t slots, cudaStream_t st) {
    if constexpr (LG > kMaxLgOdd) {
        return cudaErrorInvalidValue;
    } else {
        if (lg == LG) {
            if constexpr (odd_inner_ok<T>(RO, LG, true)) {
                return real_at<T, RO * (1 << LG)>(mode, W, tabs, N, lgL1, lgM, tw, scale, slots, st);
            } else {
                return cudaErrorInvalidValue;
            }
        }
        return real_odd_dispatch<T, RO, LG + 1>(lg, mode, W, tabs, N, lgL1, lgM, tw, scale, slots, st);
    }
}

template <typename T, int RO>
cudaError_t launch_middle_real_odd(int lg, int mode, cx<T> *W, cx<T> *tabs, uint64_t N, uint32_t lgL1, uint32_t lgM,
                                   TwTab<T> tw, T scale, uint32_t slots, cudaStream_t st) {
    return real_odd_dispatch<T, RO>(lg, mode, W, tabs, N, lgL1, lgM, tw, scale, slots, st);
}

template <typename T>
cudaError_t launch_middle_real(int ro, int lg, int mode, cx<T> *W, cx<T> *tabs, uint64_t N, uint32_t lgL1,
                               uint32_t lgM, TwTab<T> tw, T scale, uint32_t slots, cudaStream_t st) {
    if (ro == 1) {
        return by_len<kMinLgMiddle, MaxLgSplit<T>::v>(lg, [&](auto c) {
            return real_at<T, decltype(c)::value>(mode, W, tabs, N, lgL1, lgM, tw, scale, slots, st);
        });
    }
    if (ro == 3) return launch_middle_real_odd<T, 3>(lg, mode, W, tabs, N, lgL1, lgM, tw, scale, slots, st);
    if (ro == 5) return launch_middle_real_odd<T, 5>(lg, mode, W, tabs, N, lgL1, lgM, tw, scale, slots, st);
    if (ro == 9) return launch_middle_real_odd<T, 9>(lg, mode, W, tabs, N, lgL1, lgM, tw, scale, slots, st);
    return cudaErrorInvalidValue;
}

// Odd innermost lengths of one (type, RO): the plain middle pass and the split pass.
#define PA_INSTANTIATE_ODD(T, RO)                                                                               \
    template cudaError_t launch_middle_odd<T, RO>(int, int, cx<T> *, cx<T> *, uint64_t, uint32_t, TwTab<T>,     \
                                                  cx<T>, cudaStream_t);                                         \
    template cudaError_t launch_middle_split_odd<T, RO>(int, const cx<T> *, cx<T> *, uint64_t, uint32_t,        \
                                                        uint32_t, uint32_t, TwTab<T>, cudaStream_t);            \
    template cudaError_t launch_middle_real_odd<T, RO>(int, int, cx<T> *, cx<T> *, uint64_t, uint32_t, uint32_t, \
                                                       TwTab<T>, T, uint32_t, cudaStream_t);

}  // namespace pa

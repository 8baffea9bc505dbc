// pa_launch.cuh -- launcher definitions; included by the per-type .cu files.
#pragma once

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

template <typename T>
cudaError_t launch_fwd_keys(int lgLEN, const uint64_t *keys, uint32_t nkeys, uint64_t kstride, uint64_t n,
                            cx<T> *W, uint64_t L, uint32_t pairs, TwTab<T> tw, cudaStream_t st) {
    constexpr int E = Shape<T>::E, COLS = Shape<T>::COLS;
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        auto kern = k_fwd_keys<T, LEN, COLS, E>;
        constexpr size_t sb = smem_bytes<T, LEN, COLS>();
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((L / LEN) / COLS), pairs);
        kern<<<grid, COLS * LEN / E, sb, st>>>(keys, nkeys, kstride, n, W, L, tw);
        return cudaGetLastError();
    });
}

template <typename T>
cudaError_t launch_fwd_seed(int lgLEN, const uint64_t *seed, uint64_t n, uint64_t m, cx<T> *W, uint64_t L,
                            TwTab<T> tw, cudaStream_t st) {
    constexpr int E = Shape<T>::E, COLS = Shape<T>::COLS;
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        auto kern = k_fwd_seed<T, LEN, COLS, E>;
        constexpr size_t sb = smem_bytes<T, LEN, COLS>();
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((L / LEN) / COLS), 1);
        kern<<<grid, COLS * LEN / E, sb, st>>>(seed, n, m, W, L, tw);
        return cudaGetLastError();
    });
}

template <typename T>
cudaError_t launch_mid(int lgLEN, bool inverse, cx<T> *W, uint64_t L, uint32_t lgS, uint32_t pairs, TwTab<T> tw,
                       cudaStream_t st) {
    constexpr int E = Shape<T>::E, COLS = Shape<T>::COLS;
    return by_len<kMinLgStrided, kMinLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        constexpr size_t sb = smem_bytes<T, LEN, COLS>();
        const uint64_t nblk = L >> (lgLEN + lgS);
        dim3 grid((unsigned)((1ull << lgS) / COLS), (unsigned)(nblk * pairs));
        if (inverse) {
            auto kern = k_mid<T, LEN, COLS, E, true>;
            cudaError_t e = set_smem(kern, sb);
            if (e != cudaSuccess) return e;
            kern<<<grid, COLS * LEN / E, sb, st>>>(W, L, lgS, tw);
        } else {
            auto kern = k_mid<T, LEN, COLS, E, false>;
            cudaError_t e = set_smem(kern, sb);
            if (e != cudaSuccess) return e;
            kern<<<grid, COLS * LEN / E, sb, st>>>(W, L, lgS, tw);
        }
        return cudaGetLastError();
    });
}

template <typename T>
cudaError_t launch_middle(int lgLEN, int mode, cx<T> *W, cx<T> *spec, uint64_t L, uint32_t pairs, TwTab<T> tw,
                          cx<T> scale, cudaStream_t st) {
    constexpr int E = Shape<T>::E;
    return by_len<kMinLgMiddle, MaxLgMiddle<T>::v>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
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
    });
}

template <typename T>
cudaError_t launch_inv_bits(int lgLEN, const cx<T> *W, uint64_t L, uint64_t m, uint32_t nkeys,
                            const uint32_t *popc, uint32_t *margin_bits, uint64_t *out, uint64_t ostride,
                            uint32_t pairs, TwTab<T> tw, cudaStream_t st) {
    constexpr int E = Shape<T>::E, COLS = Shape<T>::COLS;
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        auto kern = k_inv_bits<T, LEN, COLS, E>;
        constexpr size_t sb = smem_bytes<T, LEN, COLS>();
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((L / LEN) / COLS), pairs);
        kern<<<grid, COLS * LEN / E, sb, st>>>(W, L, m, nkeys, popc, margin_bits, out, ostride, tw);
        return cudaGetLastError();
    });
}

#define PA_INSTANTIATE_LAUNCHERS(T)                                                                              \
    template cudaError_t launch_fwd_keys<T>(int, const uint64_t *, uint32_t, uint64_t, uint64_t, cx<T> *,        \
                                            uint64_t, uint32_t, TwTab<T>, cudaStream_t);                         \
    template cudaError_t launch_fwd_seed<T>(int, const uint64_t *, uint64_t, uint64_t, cx<T> *, uint64_t,        \
                                            TwTab<T>, cudaStream_t);                                             \
    template cudaError_t launch_mid<T>(int, bool, cx<T> *, uint64_t, uint32_t, uint32_t, TwTab<T>,               \
                                       cudaStream_t);                                                           \
    template cudaError_t launch_middle<T>(int, int, cx<T> *, cx<T> *, uint64_t, uint32_t, TwTab<T>, cx<T>,       \
                                          cudaStream_t);                                                        \
    template cudaError_t launch_inv_bits<T>(int, const cx<T> *, uint64_t, uint64_t, uint32_t, const uint32_t *,  \
                                            uint32_t *, uint64_t *, uint64_t, uint32_t, TwTab<T>, cudaStream_t);

template <typename T>
cudaError_t launch_fwd_keyseed(int lgLEN, const BlockDev *blocks, uint32_t nblocks, cx<T> *W, uint64_t L,
                               TwTab<T> tw, cudaStream_t st) {
    constexpr int E = Shape<T>::E, COLS = Shape<T>::COLS;
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        auto kern = k_fwd_keyseed<T, LEN, COLS, E>;
        constexpr size_t sb = smem_bytes<T, LEN, COLS>();
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((L / LEN) / COLS), nblocks);
        kern<<<grid, COLS * LEN / E, sb, st>>>(blocks, W, L, tw);
        return cudaGetLastError();
    });
}

template <typename T>
cudaError_t launch_middle_split(int lgLEN, const cx<T> *Wf, cx<T> *Wi, uint64_t L, uint32_t nblocks, uint32_t lgL1,
                                uint32_t lgM, TwTab<T> tw, cudaStream_t st) {
    constexpr int E = Shape<T>::E;
    return by_len<kMinLgMiddle, MaxLgSplit<T>::v>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
        auto kern = k_middle_split<T, LEN, E>;
        constexpr size_t sb = 2 * smem_bytes<T, LEN, 1>();
        cudaError_t e = set_smem(kern, sb);
        if (e != cudaSuccess) return e;
        const uint32_t R = (uint32_t)(L / LEN);
        dim3 grid(R / 2 + 1, (nblocks + 1) / 2);
        kern<<<grid, 2 * (LEN / E), sb, st>>>(Wf, Wi, L, nblocks, lgL1, lgM, tw, (T)(1.0 / (double)L));
        return cudaGetLastError();
    });
}

template <typename T>
cudaError_t launch_inv_bits_blocks(int lgLEN, const cx<T> *Wi, uint64_t L, const BlockDev *blocks, uint32_t nblocks,
                                   const uint32_t *popc, uint32_t *margin_bits, TwTab<T> tw, cudaStream_t st) {
    constexpr int E = Shape<T>::E, COLS = Shape<T>::COLS;
    return by_len<kMinLgStrided, kMaxLgStrided>(lgLEN, [&](auto c) {
        constexpr int LEN = decltype(c)::value;
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
                                               cudaStream_t);                                                   \
    template cudaError_t launch_middle_split<T>(int, const cx<T> *, cx<T> *, uint64_t, uint32_t, uint32_t,       \
                                                uint32_t, TwTab<T>, cudaStream_t);                               \
    template cudaError_t launch_inv_bits_blocks<T>(int, const cx<T> *, uint64_t, const BlockDev *, uint32_t,     \
                                                   const uint32_t *, uint32_t *, TwTab<T>, cudaStream_t);

}  // namespace pa

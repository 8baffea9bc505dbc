// pa_prep.cu -- per-key preparation: popcount and margin reset.
#include "pa_launch.h"

namespace pa {

// One CTA per key. P = popcount of the key's bits below n; it enters the
// rounding step as P mod 4 (see the encoding note in pa_kernels.cuh).
__global__ void __launch_bounds__(256)
    k_prep(const uint64_t *__restrict__ keys, uint32_t nkeys, uint64_t kstride, uint64_t n,
           uint32_t *__restrict__ popc, uint32_t *__restrict__ margin_bits) {
    const uint32_t key = blockIdx.x;
    const uint64_t *k = keys + (uint64_t)key * kstride;
    const uint64_t nw = (n + 63) >> 6;
    uint32_t acc = 0;
    for (uint64_t w = threadIdx.x; w < nw; w += blockDim.x) {
        uint64_t x = __ldg(k + w);
        if (w == nw - 1 && (n & 63)) x &= (1ull << (n & 63)) - 1ull;
        acc += (uint32_t)__popcll(x);
    }
    acc = __reduce_add_sync(0xffffffffu, acc);
    __shared__ uint32_t part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
        popc[key] = t;
        margin_bits[key] = 0u;
    }
}

cudaError_t launch_prep(const uint64_t *keys, uint32_t nkeys, uint64_t kstride, uint64_t n, uint32_t *popc,
                        uint32_t *margin_bits, cudaStream_t st) {
    if (nkeys == 0) return cudaSuccess;
    k_prep<<<nkeys, 256, 0, st>>>(keys, nkeys, kstride, n, popc, margin_bits);
    return cudaGetLastError();
}

}  // namespace pa

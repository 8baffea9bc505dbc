// pa_prep.cu -- per-key preparation: popcount and margin reset.
#include <mutex>
#include <set>
#include <utility>

#include "pa_kernels.cuh"
#include "pa_launch.h"

namespace pa {

namespace {
std::mutex g_smem_mu;
std::set<std::pair<const void *, int>> g_smem_done;
}  // namespace

bool smem_configured(const void *kernel, int device) {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    return g_smem_done.count({kernel, device}) != 0;
}

void smem_mark_configured(const void *kernel, int device) {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    g_smem_done.insert({kernel, device});
}

// Per-key state of a batch: the popcount P (accumulated by the level-1 forward
// pass, which reads every key bit; it enters the rounding step as P mod 4, see the
// encoding note in pa_kernels.cuh) and the rounding margin start at zero.
__global__ void k_zero_keys(uint32_t nkeys, uint32_t *__restrict__ popc, uint32_t *__restrict__ margin_bits) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nkeys) {
        popc[k] = 0u;
        margin_bits[k] = 0u;
    }
}

cudaError_t launch_zero_keys(uint32_t nkeys, uint32_t *popc, uint32_t *margin_bits, cudaStream_t st) {
    if (nkeys == 0) return cudaSuccess;
    k_zero_keys<<<(nkeys + 255) / 256, 256, 0, st>>>(nkeys, popc, margin_bits);
    return cudaGetLastError();
}


// One CTA per block of an uneven batch: popcount of its key (bits < n) into
// popc[id], margin[id] reset.
__global__ void __launch_bounds__(256)
    k_prep_blocks(const BlockDev *__restrict__ blocks, uint32_t *__restrict__ popc, uint32_t *__restrict__ margin_bits) {
    const BlockDev bd = blocks[blockIdx.x];
    const uint64_t nw = (bd.n + 63) >> 6;
    uint32_t acc = 0;
    for (uint64_t w = threadIdx.x; w < nw; w += blockDim.x) {
        uint64_t x = __ldg(bd.key + w);
        if (w == nw - 1 && (bd.n & 63)) x &= (1ull << (bd.n & 63)) - 1ull;
        acc += (uint32_t)__popcll(x);
    }
    acc = __reduce_add_sync(0xffffffffu, acc);
    __shared__ uint32_t part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
        popc[bd.id] = t;
        margin_bits[bd.id] = 0u;
    }
}

cudaError_t launch_prep_blocks(const BlockDev *blocks, uint32_t nblocks, uint32_t *popc, uint32_t *margin_bits,
                               cudaStream_t st) {
    if (nblocks == 0) return cudaSuccess;
    k_prep_blocks<<<nblocks, 256, 0, st>>>(blocks, popc, margin_bits);
    return cudaGetLastError();
}

}  // namespace pa

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


// One thread per block of an uneven batch: popc[id] and margin[id] start at zero
// (the level-1 key+seed pass adds the popcount of every key bit it stages).
__global__ void k_zero_blocks(const BlockDev *__restrict__ blocks, uint32_t nblocks, uint32_t *__restrict__ popc,
                              uint32_t *__restrict__ margin_bits) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nblocks) {
        const uint32_t id = blocks[b].id;
        popc[id] = 0u;
        margin_bits[id] = 0u;
    }
}

cudaError_t launch_zero_blocks(const BlockDev *blocks, uint32_t nblocks, uint32_t *popc, uint32_t *margin_bits,
                               cudaStream_t st) {
    if (nblocks == 0) return cudaSuccess;
    k_zero_blocks<<<(nblocks + 255) / 256, 256, 0, st>>>(blocks, nblocks, popc, margin_bits);
    return cudaGetLastError();
}

}  // namespace pa

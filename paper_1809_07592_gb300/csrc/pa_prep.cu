// pa_prep.cu -- per-key preparation: popcount and margin reset.
#include <mutex>
#include <cuda.h>
#include <set>
#include <utility>

#include "pa_kernels.cuh"
#include "pa_launch.h"

namespace pa {

namespace {
std::mutex g_smem_mu;
std::set<std::pair<const void *, int>> g_smem_done;
}  // namespace

bool encode_tile_map(CUtensorMap *map, const void *base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                     uint32_t box_rows) {
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<Encode>(f);
        cudaGetLastError();
    });
    if (!encode) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 8};  // bytes between rows (a multiple of 16: cols is even)
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

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

// Round every float of x[0 .. count) to `bits` explicit significand bits (round to
// nearest, ties to even, on the float's encoding), as if the values had been stored in a
// format with that significand and FP32's exponent range.
__global__ void k_round_significand(float *__restrict__ x, uint64_t count, uint32_t bits) {
    const uint32_t drop = 23u - bits;
    const uint32_t half = (1u << (drop - 1)) - 1u, mask = ~((1u << drop) - 1u);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = __float_as_uint(x[i]);
        u = (u + half + ((u >> drop) & 1u)) & mask;
        x[i] = __uint_as_float(u);
    }
}

cudaError_t launch_round_significand(float *x, uint64_t count, uint32_t bits, cudaStream_t st) {
    if (bits == 0 || bits >= 23 || count == 0) return cudaSuccess;
    k_round_significand<<<1184, 256, 0, st>>>(x, count, bits);
    return cudaGetLastError();
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

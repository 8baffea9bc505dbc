// pa_internal.h -- helpers shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

// Records "what: cuda error string" as the calling thread's last CUDA error and returns PA_ECUDA.
int pa_internal_cuda_fail(cudaError_t e, const char *what);

// Device twiddle tables of the length-L transform for a pa_dtype_t (cudaMalloc'd; caller frees):
// the two-level table hi/lo split at B, and the stage table fine of length F (F divides L).
int pa_internal_twiddles(uint64_t L, uint32_t F, int dtype, void **hi, void **lo, uint32_t *B, void **fine);

#include "pa.h"

namespace pa {

// Transform geometry: length L = lgL-free description
//   L = 2^lg1 * 2^lgM * (ro * 2^lgI)
// strided level-1 pass 2^lg1, optional middle strided pass 2^lgM (lgM = 0: none),
// innermost pass ro * 2^lgI (ro in {1, 3, 5, 9}). F = lcm of the pass lengths is
// the length of the stage-twiddle table.
struct Geometry {
    uint64_t L = 0;
    int lg1 = 0, lgM = 0, ro = 1, lgI = 0;
    uint32_t inner() const { return (uint32_t)ro << lgI; }
    uint32_t F() const {
        int m = lg1 > lgM ? lg1 : lgM;
        if (lgI > m) m = lgI;
        return (uint32_t)ro << m;
    }
};

// Every valid split of length L for the arithmetic `dtype` (split = the
// innermost pass is the two-row Eq. 5-10 kernel of the uneven batch).
std::vector<Geometry> geometry_candidates(uint64_t L, pa_dtype_t dtype, bool split);
// The preferred split of L (two levels when possible, innermost length near 2^12), or L = 0.
Geometry default_geometry(uint64_t L, pa_dtype_t dtype, bool split);
// The smallest supported transform length >= max(need, 2^12): ro * 2^k with ro in {1, 3, 5, 9}
// (ro = 1 only for the exact transform), together with its default split.
Geometry choose_geometry(uint64_t need, pa_dtype_t dtype, bool split);

}  // namespace pa

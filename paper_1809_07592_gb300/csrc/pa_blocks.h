// pa_blocks.h -- per-length-class chains of the uneven batch, shared by the
// batch planner (pa_uneven.cu) and the serving loop (pa_server.cu). Internal:
// not part of the C ABI.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "pa.h"
#include "pa_internal.h"

namespace pa {
struct BlockDev;
namespace blocks {

// Everything one class's chain touches (device pointers).
struct ClassRun {
    Geometry geo;                        // transform length and pass split
    const BlockDev *d_blocks = nullptr;  // nb descriptors
    uint32_t nb = 0;
    void *Wf = nullptr;    // complex: nb slots of L values; NTT: one slot
    void *Wi = nullptr;    // complex: ceil(nb/2) slots
    void *spec = nullptr;  // NTT: one seed-spectrum slot
    const void *tw_hi = nullptr, *tw_lo = nullptr;
    uint32_t B = 0;
    const void *tw_fine = nullptr;  // stage twiddles, length geo.F()
};

// Transform length of a block of an uneven batch / the serving loop.
uint64_t class_length(uint64_t n, uint64_t m, pa_dtype_t dtype);

// Bytes of device scratch one block of transform length L needs in a class run.
size_t scratch_per_block(uint64_t L, pa_dtype_t dtype);

// Launch the chain of one class on `st`. Complex modes (Eq. 5-10 split): popcounts
// and margins of block d_blocks[i] go to popc[id], marg[id]. NTT mode: host copies of
// the descriptors (`hb`, indexed by `ids`) drive one exact chain per block.
int run_complex(pa_dtype_t dtype, const ClassRun &c, uint32_t *popc, uint32_t *marg, cudaStream_t st);
int run_ntt(const ClassRun &c, const pa_block_desc_t *hb, const uint32_t *ids, uint32_t *popc, uint32_t *marg,
            cudaStream_t st);

// Candidate splits of a class length, the tuned split from the cache (if any), and a default.
std::vector<Geometry> candidates(uint64_t L, pa_dtype_t dtype);
bool cached_split(uint64_t L, pa_dtype_t dtype, Geometry *out);
void store_split(const Geometry &g, pa_dtype_t dtype);
Geometry default_split(uint64_t L, pa_dtype_t dtype);

}  // namespace blocks
}  // namespace pa

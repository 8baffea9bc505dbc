// pa_blocks.h -- per-length-class chains of the uneven batch, shared by the
// batch planner (pa_uneven.cu) and the serving loop (pa_server.cu). Internal:
// not part of the C ABI.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "pa.h"

namespace pa {
struct BlockDev;
namespace blocks {

// Pass split of a class: strided level-1 length, middle strided length (0: two
// levels) and innermost length, all log2.
struct Split {
    int lg1 = 0, lgM = 0, lgI = 0;
};

// Everything one class's chain touches (device pointers).
struct ClassRun {
    int lgL = 0;
    uint64_t L = 0;
    Split sp;
    const BlockDev *d_blocks = nullptr;  // nb descriptors
    uint32_t nb = 0;
    void *Wf = nullptr;    // complex: nb slots of L values; NTT: one slot
    void *Wi = nullptr;    // complex: ceil(nb/2) slots
    void *spec = nullptr;  // NTT: one seed-spectrum slot
    const void *tw_hi = nullptr, *tw_lo = nullptr;
    uint32_t B = 0;
};

// Bytes of device scratch one block of transform length 2^lgL needs in a class run.
size_t scratch_per_block(int lgL, pa_dtype_t dtype);

// Launch the chain of one class on `st`. Complex modes (Eq. 5-10 split): popcounts
// and margins of block d_blocks[i] go to popc[id], marg[id]. NTT mode: host copies of
// the descriptors (`hb`, indexed by `ids`) drive one exact chain per block.
int run_complex(pa_dtype_t dtype, const ClassRun &c, uint32_t *popc, uint32_t *marg, cudaStream_t st);
int run_ntt(const ClassRun &c, const pa_block_desc_t *hb, const uint32_t *ids, uint32_t *popc, uint32_t *marg,
            cudaStream_t st);

// Candidate splits, the tuned split from the cache (if any), and a default.
std::vector<Split> candidates(int lgL, pa_dtype_t dtype);
bool cached_split(int lgL, pa_dtype_t dtype, Split *out);
void store_split(int lgL, pa_dtype_t dtype, const Split &s);
Split default_split(int lgL, pa_dtype_t dtype);

// log2 of the transform length of a block: max(12, ceil(log2(n + m - 1))).
int lg_length(uint64_t n, uint64_t m);

}  // namespace blocks
}  // namespace pa

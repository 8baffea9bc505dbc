// pa_zp.cu -- modular (NTT, p = 2^64 - 2^32 + 1) instances of the pass kernels and launchers.
#include "pa_launch.cuh"

namespace pa {
PA_INSTANTIATE_LAUNCHERS(Zp)
}  // namespace pa

// pa_f32.cu -- single-precision instances of the pass kernels and launchers.
#include "pa_launch.cuh"

namespace pa {
PA_INSTANTIATE_LAUNCHERS(float)
PA_INSTANTIATE_UNEVEN(float)
}  // namespace pa

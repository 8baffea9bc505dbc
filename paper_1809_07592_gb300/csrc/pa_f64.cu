// pa_f64.cu -- double-precision instances of the pass kernels and launchers.
#include "pa_launch.cuh"

namespace pa {
PA_INSTANTIATE_LAUNCHERS(double)
PA_INSTANTIATE_UNEVEN(double)
}  // namespace pa

// pa_f32_r5.cu -- single-precision innermost passes of length 5 * 2^lg (smooth transform lengths).
#include "pa_launch.cuh"

namespace pa {
PA_INSTANTIATE_ODD(float, 5)
}  // namespace pa

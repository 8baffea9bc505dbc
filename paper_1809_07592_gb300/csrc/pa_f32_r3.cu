// pa_f32_r3.cu -- single-precision innermost passes of length 3 * 2^lg (smooth transform lengths).
#include "pa_launch.cuh"

namespace pa {
PA_INSTANTIATE_ODD(float, 3)
}  // namespace pa

// pa_f64_r5.cu -- double-precision innermost passes of length 5 * 2^lg (smooth transform lengths).
#include "pa_launch.cuh"

namespace pa {
PA_INSTANTIATE_ODD(double, 5)
}  // namespace pa

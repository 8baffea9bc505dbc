// pa_f64_r9.cu -- double-precision innermost passes of length 9 * 2^lg (smooth transform lengths).
#include "pa_launch.cuh"

namespace pa {
PA_INSTANTIATE_ODD(double, 9)
}  // namespace pa

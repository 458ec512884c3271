// Kernel instantiations for 3D, arithmetic float, population storage __half.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS(ops_d3_f16, 3, float, __half)
}  // namespace gpflbm

// Kernel instantiations for 3D, arithmetic float, population storage float.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS(ops_d3_fp32, 3, float, float)
}  // namespace gpflbm

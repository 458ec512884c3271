// Kernel instantiations for 2D, arithmetic float, population storage float.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS(ops_d2_fp32, 2, float, float)
}  // namespace gpflbm

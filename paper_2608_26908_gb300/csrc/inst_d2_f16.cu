// Kernel instantiations for 2D, arithmetic float, population storage __half.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS(ops_d2_f16, 2, float, __half)
}  // namespace gpflbm

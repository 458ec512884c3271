// Kernel instantiations for 2D, arithmetic float, population storage __nv_bfloat16.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS(ops_d2_bf16, 2, float, __nv_bfloat16)
}  // namespace gpflbm

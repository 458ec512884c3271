// Kernel instantiations for 3D, arithmetic float, population storage __nv_bfloat16.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS(ops_d3_bf16, 3, float, __nv_bfloat16)
}  // namespace gpflbm

// Kernel instantiations for 3D on D3Q27, arithmetic float, population storage float.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS_Q(ops_d3q27_fp32, 3, 27, float, float)
}  // namespace gpflbm

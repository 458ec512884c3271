// Kernel instantiations for 3D on D3Q27, arithmetic double, population storage double.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS_Q(ops_d3q27_fp64, 3, 27, double, double)
}  // namespace gpflbm

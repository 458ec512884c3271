// Kernel instantiations for 3D, arithmetic double, population storage double.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS(ops_d3_fp64, 3, double, double)
}  // namespace gpflbm

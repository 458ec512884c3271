// Kernel instantiations for 2D, arithmetic double, population storage double.
#include "gpflbm_ops.cuh"

namespace gpflbm {
GPFLBM_DEFINE_OPS(ops_d2_fp64, 2, double, double)
}  // namespace gpflbm

// Launchers of the 2D two-phase adjoint kernels (adjoint2d.cuh), gathered in
// a table of plain function pointers for the C-ABI layer.  Buffers are in
// the internal layout (padded row pitch) and hold the arithmetic type.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace gpflbm {

struct AdjStepIO {
  const void* s0;   // S^n: phi_1, mu, f - w (9 planes)
  const void* mu0;
  const void* d0;
  const void* s1;   // S^{n+1}: phi_1, mu
  const void* mu1;
  const void* ls1;  // adjoint of S^{n+1}
  const void* lmu1;
  const void* ld1;
  void* ls0;        // adjoint of S^n (written)
  void* lmu0;
  void* ld0;
  double* gacc;     // 3 FP64 planes, accumulated
  const double* clock;  // time of step n (device)
};

struct AdjOps {
  size_t real_size;
  // opts the step kernel in to its dynamic shared memory
  cudaError_t (*configure)();
  // lambda of the final state from w_frac mean h_1; clears gacc
  cudaError_t (*init)(const void* P, const void* s, double w_frac, void* ls, void* lmu, void* ld,
                      double* gacc, cudaStream_t st);
  // adds the soft-argmax tip term to ls and writes tip (device double)
  cudaError_t (*tip)(const void* P, const void* s, int x0, int y0, double kappa, double w_tip, void* ls,
                     double* tip, cudaStream_t st);
  // fixed-order partial sums of h_1 over the cells (blocks partials)
  cudaError_t (*frac)(const void* P, const void* s, double* partial, int blocks, cudaStream_t st);
  // one adjoint step lambda^{n+1} -> lambda^n (one launch)
  cudaError_t (*step)(const void* P, const AdjStepIO& io, cudaStream_t st);
  // fixed-order partial sums of an FP64 plane over the cells
  cudaError_t (*sum)(const void* P, const double* v, double* partial, int blocks, cudaStream_t st);
  // one plane to the exchange layout (x fastest, no padding)
  cudaError_t (*export_plane)(const void* P, const void* src, void* dst, cudaStream_t st);
  // one plane from the exchange layout into the internal layout
  cudaError_t (*import_plane)(const void* P, const void* src, void* dst, cudaStream_t st);
};

// Table for FP64 (fp64 != 0) or FP32 arithmetic.
const AdjOps* adjoint_ops(int fp64);

}  // namespace gpflbm

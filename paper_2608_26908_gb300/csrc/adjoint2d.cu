// Launchers of the 2D two-phase adjoint step and of the objective kernels.
#include "adjoint2d.cuh"
#include "adjoint_ops.h"

namespace gpflbm {
namespace {

constexpr int kThreads = 256;

template <class Real>
unsigned cell_blocks(const DevParams<Real>& P) {
  const long long cells = (long long)P.n[0] * P.n[1];
  return (unsigned)((cells + kThreads - 1) / kThreads);
}

template <class Real>
struct AdjImpl {
  static const DevParams<Real>& par(const void* p) { return *static_cast<const DevParams<Real>*>(p); }

  static cudaError_t init(const void* p, const void* s, double w_frac, void* ls, void* lmu, void* ld,
                          double* gacc, cudaStream_t st) {
    const DevParams<Real>& P = par(p);
    adj_init_kernel<Real><<<cell_blocks(P), kThreads, 0, st>>>(
        P, static_cast<const Real*>(s), (Real)w_frac, static_cast<Real*>(ls), static_cast<Real*>(lmu),
        static_cast<Real*>(ld), gacc);
    return cudaGetLastError();
  }

  static cudaError_t tip(const void* p, const void* s, int x0, int y0, double kappa, double w_tip, void* ls,
                         double* tip_out, cudaStream_t st) {
    adj_tip_kernel<Real><<<1, 256, 0, st>>>(par(p), static_cast<const Real*>(s), x0, y0, kappa, w_tip,
                                            static_cast<Real*>(ls), tip_out);
    return cudaGetLastError();
  }

  static cudaError_t frac(const void* p, const void* s, double* partial, int blocks, cudaStream_t st) {
    adj_frac_kernel<Real><<<blocks, kRedThreads, 0, st>>>(par(p), static_cast<const Real*>(s), partial);
    return cudaGetLastError();
  }

  static cudaError_t configure() {
    return cudaFuncSetAttribute(adj2d_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Adj2D<Real>::bytes);
  }

  static cudaError_t step(const void* p, const AdjStepIO& v, cudaStream_t st) {
    using S = Adj2D<Real>;
    const DevParams<Real>& P = par(p);
    AdjIO<Real> io;
    io.s0 = static_cast<const Real*>(v.s0);
    io.mu0 = static_cast<const Real*>(v.mu0);
    io.d0 = static_cast<const Real*>(v.d0);
    io.s1 = static_cast<const Real*>(v.s1);
    io.mu1 = static_cast<const Real*>(v.mu1);
    io.ls1 = static_cast<const Real*>(v.ls1);
    io.lmu1 = static_cast<const Real*>(v.lmu1);
    io.ld1 = static_cast<const Real*>(v.ld1);
    io.ls0 = static_cast<Real*>(v.ls0);
    io.lmu0 = static_cast<Real*>(v.lmu0);
    io.ld0 = static_cast<Real*>(v.ld0);
    io.gacc = v.gacc;
    io.clock = v.clock;
    // programmatic dependent launch: this step's prologue (stored states
    // only) overlaps the previous step's last CTAs; the kernel waits for
    // the previous step before it touches lambda or gacc
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((P.n[0] + S::OX - 1) / S::OX, (P.n[1] + S::OY - 1) / S::OY);
    cfg.blockDim = dim3(S::NT);
    cfg.dynamicSmemBytes = S::bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, adj2d_kernel<Real>, P, io);
  }

  static cudaError_t sum(const void* p, const double* v, double* partial, int blocks, cudaStream_t st) {
    adj_sum_kernel<Real><<<blocks, kRedThreads, 0, st>>>(par(p), v, partial);
    return cudaGetLastError();
  }

  static cudaError_t export_plane(const void* p, const void* src, void* dst, cudaStream_t st) {
    const DevParams<Real>& P = par(p);
    adj_export_kernel<Real><<<cell_blocks(P), kThreads, 0, st>>>(P, static_cast<const Real*>(src),
                                                                 static_cast<Real*>(dst));
    return cudaGetLastError();
  }

  static cudaError_t import_plane(const void* p, const void* src, void* dst, cudaStream_t st) {
    const DevParams<Real>& P = par(p);
    adj_import_kernel<Real><<<cell_blocks(P), kThreads, 0, st>>>(P, static_cast<const Real*>(src),
                                                                 static_cast<Real*>(dst));
    return cudaGetLastError();
  }

  static const AdjOps* table() {
    static const AdjOps t = {sizeof(Real), configure, init, tip, frac, step, sum, export_plane, import_plane};
    return &t;
  }
};

}  // namespace

const AdjOps* adjoint_ops(int fp64) {
  return fp64 ? AdjImpl<double>::table() : AdjImpl<float>::table();
}

}  // namespace gpflbm

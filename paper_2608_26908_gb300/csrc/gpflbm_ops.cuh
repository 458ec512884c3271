// Launchers of the device kernels for one (dimension, phases, solutes,
// arithmetic type, storage type) combination, gathered in a table of plain
// function pointers so that the C-ABI layer dispatches at run time.
#pragma once

#include <cuda_runtime.h>

#include "gpflbm_kernels.cuh"
#include "step2d.cuh"
#include "step3d.cuh"
#include "step3d_liquid.cuh"

namespace gpflbm {

struct StepIO {
  const void* phi_in;
  void* phi_out;
  const void* mu_in;
  void* mu_out;
  const void* f_in;
  void* f_out;
  const double* clock_in;
  double* clock_out;
  const unsigned char* flags_in;  // 3D: liquid flag per tile of the input state
  unsigned char* flags_out;       // ... of the output state
};

struct FieldsIO {
  const void* phi;
  const void* mu;
  const void* f;
  const double* clock;
  void* o_phi;
  void* o_mu;
  void* o_c;
  void* o_f;
  void* o_rho;
  void* o_u;
  void* o_dev;
};

struct Ops {
  int D, NP, NC, Q;
  size_t real_size, store_size;
  int stored_phi_planes;
  // 3D: launches of one step when liquid tiles take their own path (1: one
  // launch runs both paths; 2: the general kernel, then the liquid kernel)
  int liquid_step_launches;
  // opts the step kernels in to their dynamic shared memory (once per process)
  cudaError_t (*configure)();
  // one time step S^n -> S^{n+1}: one fused launch
  cudaError_t (*step)(const void* params, const StepIO& io, cudaStream_t s);
  // exchange planes (Real) -> stored state; src_f may be null (rest)
  cudaError_t (*load)(const void* params, const void* src_phi, const void* src_mu,
                      const void* src_f, void* phi, void* mu, void* f, cudaStream_t s);
  // the whole state (src_f may be null) and the step counters (clock_b may
  // be null), in one launch
  cudaError_t (*load_state)(const void* params, const void* src_phi, const void* src_mu,
                            const void* src_f, void* phi, void* mu, void* f, double* clock_a,
                            double* clock_b, double t0, cudaStream_t s);
  cudaError_t (*fields)(const void* params, const FieldsIO& io, cudaStream_t s);
  cudaError_t (*invariants)(const InvParams& p, const void* phi, const void* mu, const void* f,
                            double* partial, int blocks, double* out, cudaStream_t s);
  // 3D: the liquid flag of every tile of a state (its phi buffer); 2D: nothing
  cudaError_t (*classify)(const void* params, const void* phi, unsigned char* flags, cudaStream_t s);
};

// Grid of the exchange kernels (state load, field write-back): two CTAs of
// 256 threads per SM in a grid-stride loop.  That keeps enough accesses in
// flight for the host link and for HBM, and leaves room on every SM for the
// other of the two, which may run at the same time on another stream.
inline unsigned exchange_blocks(long long items, int threads) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        v > 0)
      sms = v;
    else
      return (unsigned)((items + threads - 1) / threads);  // one item per thread
  }
  const long long need = (items + threads - 1) / threads;
  return (unsigned)(need < 2LL * sms ? need : 2LL * sms);
}

// QQ: lattice size (0 = D2Q9 in 2D, D3Q19 in 3D; 27 = D3Q27).
// EXT: the step kernels of the extended model -- turned crystal axes and
// temperature-dependent equilibrium compositions (a separate table, so that
// the plain kernels are not touched).
template <int D, int NP, int NC, class Real, class Store, int QQ = 0, bool EXT = false>
struct Impl {
  static constexpr int Q = QQ ? QQ : (D == 2 ? 9 : 19);

  using SZ = Step2D<NP, NC, Real, Store>;
  using S3 = Step3D<NP, NC, Real, Store, (D == 3 ? Q : 19)>;
  using SL = Liquid3D<NP, NC, Real, Store, (D == 3 ? Q : 19), EXT>;
  // 3D: dynamic shared memory of step3d_kernel (both paths when it runs both)
  static constexpr size_t step3d_bytes = !S3::ONE_LAUNCH ? S3::bytes : (S3::bytes > SL::bytes ? S3::bytes : SL::bytes);

  static cudaError_t configure() {
    cudaError_t e;
    if constexpr (D == 2) {
      e = cudaFuncSetAttribute(step2d_kernel<NP, NC, Real, Store, false, EXT>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SZ::bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step2d_kernel<NP, NC, Real, Store, true, EXT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SZ::bytes);
    } else {
      e = cudaFuncSetAttribute(step3d_kernel<NP, NC, Real, Store, false, Q, EXT>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step3d_bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step3d_kernel<NP, NC, Real, Store, true, Q, EXT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step3d_bytes);
      if constexpr (!S3::ONE_LAUNCH) {
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(step3d_liquid_kernel<NP, NC, Real, Store, Q, EXT>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SL::bytes);
      }
    }
    return e;
  }

  static cudaError_t step_fused(const void* params, const StepIO& io, cudaStream_t s) {
    const DevParams<Real>& P = *static_cast<const DevParams<Real>*>(params);
    if constexpr (D == 2) {
      const dim3 grid((P.n[0] + SZ::OX - 1) / SZ::OX, (P.n[1] + SZ::OY - 1) / SZ::OY);
      const Step2DIO sio = {io.phi_in, io.phi_out, io.mu_in, io.mu_out,
                            io.f_in,   io.f_out,   io.clock_in, io.clock_out};
      if (P.shrink)
        step2d_kernel<NP, NC, Real, Store, true, EXT><<<grid, SZ::NT, SZ::bytes, s>>>(P, sio);
      else
        step2d_kernel<NP, NC, Real, Store, false, EXT><<<grid, SZ::NT, SZ::bytes, s>>>(P, sio);
    } else {
      // the tiling (twice over in z when one launch takes both passes)
      const unsigned gz = (P.v_hi - P.v_lo + S3::ZS - 1) / S3::ZS;
      const dim3 grid((P.n[0] + S3::OX - 1) / S3::OX, (P.n[1] + S3::OY - 1) / S3::OY,
                      S3::ONE_LAUNCH && P.liq_dispatch ? 2 * gz : gz);
      const Step3DIO sio = {io.phi_in, io.phi_out, io.mu_in,    io.mu_out,    io.f_in,
                            io.f_out,  io.clock_in, io.clock_out, io.flags_in, io.flags_out};
      if (P.shrink)
        step3d_kernel<NP, NC, Real, Store, true, Q, EXT><<<grid, S3::NT, step3d_bytes, s>>>(P, sio);
      else
        step3d_kernel<NP, NC, Real, Store, false, Q, EXT><<<grid, S3::NT, step3d_bytes, s>>>(P, sio);
      // the tiles whose reach is pure liquid (step3d_kernel returned there)
      if constexpr (!S3::ONE_LAUNCH) {
        if (P.liq_dispatch)
          step3d_liquid_kernel<NP, NC, Real, Store, Q, EXT><<<grid, SL::NT, SL::bytes, s>>>(P, sio);
      }
    }
    return cudaGetLastError();
  }

  static cudaError_t step(const void* params, const StepIO& io, cudaStream_t s) {
    return step_fused(params, io, s);
  }

  static cudaError_t load(const void* params, const void* src_phi, const void* src_mu,
                          const void* src_f, void* phi, void* mu, void* f, cudaStream_t s) {
    const DevParams<Real>& P = *static_cast<const DevParams<Real>*>(params);
    const long long cells = (long long)P.n[0] * P.n[1] * P.n[2];
    const int threads = 256;
    const unsigned blocks = (unsigned)((cells + threads - 1) / threads);
    if (src_phi)
      load_phi_kernel<NP, Real, Real><<<blocks, threads, 0, s>>>(
          cells, P.n[0], P.px, P.plane, static_cast<const Real*>(src_phi), static_cast<Real*>(phi));
    if (src_mu)
      load_mu_kernel<NC, Real, Real><<<blocks, threads, 0, s>>>(
          cells, P.n[0], P.px, P.plane, static_cast<const Real*>(src_mu), static_cast<Real*>(mu));
    load_f_kernel<Q, Store, Real><<<blocks, threads, 0, s>>>(
        cells, P.n[0], P.px, P.plane, static_cast<const Real*>(src_f), static_cast<Store*>(f));
    return cudaGetLastError();
  }

  static cudaError_t load_state(const void* params, const void* src_phi, const void* src_mu,
                                const void* src_f, void* phi, void* mu, void* f, double* clock_a,
                                double* clock_b, double t0, cudaStream_t s) {
    const DevParams<Real>& P = *static_cast<const DevParams<Real>*>(params);
    const long long cells = (long long)P.n[0] * P.n[1] * P.n[2];
    constexpr int V = 16 / (int)sizeof(Real);  // one 16-byte word of each source plane
    auto al16 = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const bool vec = P.n[0] % V == 0 && al16(src_phi) && al16(src_mu) && al16(src_f);
    const int threads = 256;
    const long long items = vec ? cells / V : cells;
    const unsigned blocks = exchange_blocks(items, threads);
    const Real* sp = static_cast<const Real*>(src_phi);
    const Real* sm = static_cast<const Real*>(src_mu);
    const Real* sf = static_cast<const Real*>(src_f);
    if (vec)
      load_state_kernel<NP, NC, Q, Real, Store, V><<<blocks, threads, 0, s>>>(
          cells, P.n[0], P.px, P.plane, sp, sm, sf, static_cast<Real*>(phi), static_cast<Real*>(mu),
          static_cast<Store*>(f), clock_a, clock_b, t0);
    else
      load_state_kernel<NP, NC, Q, Real, Store, 1><<<blocks, threads, 0, s>>>(
          cells, P.n[0], P.px, P.plane, sp, sm, sf, static_cast<Real*>(phi), static_cast<Real*>(mu),
          static_cast<Store*>(f), clock_a, clock_b, t0);
    return cudaGetLastError();
  }

  static cudaError_t fields(const void* params, const FieldsIO& io, cudaStream_t s) {
    const DevParams<Real>& P = *static_cast<const DevParams<Real>*>(params);
    const long long cells = (long long)P.n[0] * P.n[1] * P.n[2];
    const int threads = 256;
    const unsigned blocks = exchange_blocks(cells, threads);
    fields_kernel<D, Q, NP, NC, Real, Store, Real><<<blocks, threads, 0, s>>>(
        P, static_cast<const Real*>(io.phi), static_cast<const Real*>(io.mu),
        static_cast<const Store*>(io.f), io.clock, static_cast<Real*>(io.o_phi),
        static_cast<Real*>(io.o_mu), static_cast<Real*>(io.o_c), static_cast<Real*>(io.o_f),
        static_cast<Real*>(io.o_rho), static_cast<Real*>(io.o_u), static_cast<Real*>(io.o_dev));
    return cudaGetLastError();
  }

  static cudaError_t classify(const void* params, const void* phi, unsigned char* flags, cudaStream_t s) {
    if constexpr (D == 3) {
      const DevParams<Real>& P = *static_cast<const DevParams<Real>*>(params);
      const dim3 grid((P.n[0] + S3::OX - 1) / S3::OX, (P.n[1] + S3::OY - 1) / S3::OY, P.v_hi - P.v_lo);
      liquid_flags_kernel<NP, Real><<<grid, 128, 0, s>>>(P, static_cast<const Real*>(phi), flags);
      return cudaGetLastError();
    } else {
      (void)params;
      (void)phi;
      (void)flags;
      (void)s;
      return cudaSuccess;
    }
  }

  static cudaError_t invariants(const InvParams& p, const void* phi, const void* mu, const void* f,
                                double* partial, int blocks, double* out, cudaStream_t s) {
    invariants_kernel<Q, NP, NC, Real, Store><<<blocks, kRedThreads, 0, s>>>(
        p, static_cast<const Real*>(phi), static_cast<const Real*>(mu),
        static_cast<const Store*>(f), partial);
    invariants_finish_kernel<NC + 3><<<1, 32, 0, s>>>(partial, blocks, out);
    return cudaGetLastError();
  }

  static const Ops* table() {
    static const Ops ops = {D,
                            NP,
                            NC,
                            Q,
                            sizeof(Real),
                            sizeof(Store),
                            PhiStore<NP>::NS,
                            D == 3 && !S3::ONE_LAUNCH ? 2 : 1,
                            &Impl::configure,
                            &Impl::step,
                            &Impl::load,
                            &Impl::load_state,
                            &Impl::fields,
                            &Impl::invariants,
                            &Impl::classify};
    return &ops;
  }
};

// One function per (dimension, precision) translation unit.  Each instance
// file compiles twice: with GPFLBM_EXT = 0 the plain kernels, with
// GPFLBM_EXT = 1 those of the extended model, whose table function is NAME_ext.
#define GPFLBM_DECLARE_OPS(NAME)  \
  const Ops* NAME(int NP, int NC); \
  const Ops* NAME##_ext(int NP, int NC);
GPFLBM_DECLARE_OPS(ops_d2_fp64)
GPFLBM_DECLARE_OPS(ops_d2_fp32)
GPFLBM_DECLARE_OPS(ops_d2_f16)
GPFLBM_DECLARE_OPS(ops_d2_bf16)
GPFLBM_DECLARE_OPS(ops_d3_fp64)
GPFLBM_DECLARE_OPS(ops_d3_fp32)
GPFLBM_DECLARE_OPS(ops_d3_f16)
GPFLBM_DECLARE_OPS(ops_d3_bf16)
GPFLBM_DECLARE_OPS(ops_d3q27_fp64)  // D3Q27 (FP64 and FP32 arithmetic and storage)
GPFLBM_DECLARE_OPS(ops_d3q27_fp32)

#ifndef GPFLBM_EXT
#define GPFLBM_EXT 0
#endif
#if GPFLBM_EXT
#define GPFLBM_OPS_NAME(NAME) NAME##_ext
#else
#define GPFLBM_OPS_NAME(NAME) NAME
#endif

#define GPFLBM_IMPL(DIM, NP_, NC_, QQ, REAL, STORE) Impl<DIM, NP_, NC_, REAL, STORE, QQ, (GPFLBM_EXT != 0)>
#define GPFLBM_DEFINE_OPS_Q(NAME, DIM, QQ, REAL, STORE)                               \
  const Ops* GPFLBM_OPS_NAME(NAME)(int NP, int NC) {                                  \
    if (NP == 2 && NC == 1) return GPFLBM_IMPL(DIM, 2, 1, QQ, REAL, STORE)::table();  \
    if (NP == 2 && NC == 2) return GPFLBM_IMPL(DIM, 2, 2, QQ, REAL, STORE)::table();  \
    if (NP == 3 && NC == 1) return GPFLBM_IMPL(DIM, 3, 1, QQ, REAL, STORE)::table();  \
    if (NP == 3 && NC == 2) return GPFLBM_IMPL(DIM, 3, 2, QQ, REAL, STORE)::table();  \
    if (NP == 4 && NC == 1) return GPFLBM_IMPL(DIM, 4, 1, QQ, REAL, STORE)::table();  \
    if (NP == 4 && NC == 2) return GPFLBM_IMPL(DIM, 4, 2, QQ, REAL, STORE)::table();  \
    return nullptr;                                                                   \
  }
#define GPFLBM_DEFINE_OPS(NAME, DIM, REAL, STORE) GPFLBM_DEFINE_OPS_Q(NAME, DIM, 0, REAL, STORE)

}  // namespace gpflbm

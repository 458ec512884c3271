// Device building blocks shared by the step kernels (step2d.cuh,
// step3d.cuh): lattice tables (D2Q9 in the paper's numbering, D3Q19), the
// population storage codec, the run-time parameters, the interpolation and
// gradient-energy functions of the phase field, the Gibbs-simplex
// projection; and the state I/O and fixed-order invariants kernels.
// Populations are kept as the deviation d_k = f_k - w_k so that FP32 keeps
// the small momentum sum_k c_k d_k to full relative precision; with 16-bit
// storage the deviation is the stored quantity.  No tensor cores: the step
// is a bandwidth- and issue-bound stencil, not a contraction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace gpflbm {

constexpr int kWall = 1;

// ------------------------------------------------------------------ lattices
// D2Q9 in the numbering of the paper's lattice figure; D3Q19 = rest, the six
// faces (+x,-x,+y,-y,+z,-z) and the twelve edges, each direction followed by
// its opposite.
template <int Q>
struct Lattice;

template <>
struct Lattice<9> {
  static constexpr int D = 2;
  __host__ __device__ static constexpr int c(int k, int a) {
    return a == 0   ? ((k == 1 || k == 5 || k == 8) ? 1 : ((k == 3 || k == 6 || k == 7) ? -1 : 0))
           : a == 1 ? ((k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0))
                    : 0;
  }
  __host__ __device__ static constexpr int opp(int k) {
    return k == 0 ? 0 : (k < 5 ? ((k + 1) % 4) + 1 : ((k - 3) % 4) + 5);
  }
  __host__ __device__ static constexpr double w(int k) {
    return k == 0 ? 4.0 / 9.0 : (k < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

template <>
struct Lattice<19> {
  static constexpr int D = 3;
  __host__ __device__ static constexpr int c(int k, int a) {
    // faces: k = 1..6 -> axis (k-1)/2, sign + for odd k
    // edges: e = k-7, axis pair e/4 in {(x,y), (x,z), (y,z)}, signs by e%4:
    //        (+,+), (-,-), (+,-), (-,+)
    return k == 0 ? 0
           : k < 7
               ? ((k - 1) / 2 == a ? ((k & 1) ? 1 : -1) : 0)
               : edge_c(k - 7, a);
  }
  __host__ __device__ static constexpr int edge_c(int e, int a) {
    return (a == first_axis(e / 4)) ? ((e % 4 == 0 || e % 4 == 2) ? 1 : -1)
           : (a == second_axis(e / 4)) ? ((e % 4 == 0 || e % 4 == 3) ? 1 : -1)
                                       : 0;
  }
  __host__ __device__ static constexpr int first_axis(int p) { return p == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int second_axis(int p) { return p == 0 ? 1 : 2; }
  __host__ __device__ static constexpr int opp(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }
  __host__ __device__ static constexpr double w(int k) {
    return k == 0 ? 1.0 / 3.0 : (k < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

// D3Q27: the D3Q19 directions, then the eight corners (+-1, +-1, +-1):
// c = sign * (+,+,+), (+,+,-), (+,-,+), (-,+,+) for corner pair p = 0..3,
// sign + for the first of the pair and - for its opposite.
template <>
struct Lattice<27> {
  static constexpr int D = 3;
  __host__ __device__ static constexpr int c(int k, int a) {
    return k < 19 ? Lattice<19>::c(k, a) : corner_c(k - 19, a);
  }
  __host__ __device__ static constexpr int corner_c(int e, int a) {
    return ((e / 2 != 0 && a == 3 - e / 2) ? -1 : 1) * ((e & 1) ? -1 : 1);
  }
  __host__ __device__ static constexpr int opp(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }
  __host__ __device__ static constexpr double w(int k) {
    return k == 0 ? 8.0 / 27.0 : (k < 7 ? 2.0 / 27.0 : (k < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
  }
};

// ------------------------------------------------------------------ storage codec
// Population deviation d = f - w in the storage type.  FP16 scales by 2^10
// so that deviations down to 6e-8 stay normal; BF16 stores d as is.
template <class Store>
struct Codec;
template <>
struct Codec<double> {
  __device__ static double load(double s) { return s; }
  __device__ static double put(double v) { return v; }
};
template <>
struct Codec<float> {
  __device__ static float load(float s) { return s; }
  __device__ static float put(float v) { return v; }
};
template <>
struct Codec<__half> {
  __device__ static float load(__half s) { return __half2float(s) * (1.0f / 1024.0f); }
  __device__ static __half put(float v) { return __float2half_rn(v * 1024.0f); }
};
template <>
struct Codec<__nv_bfloat16> {
  __device__ static float load(__nv_bfloat16 s) { return __bfloat162float(s); }
  __device__ static __nv_bfloat16 put(float v) { return __float2bfloat16_rn(v); }
};

// ------------------------------------------------------------------ parameters
// All per-run constants, in the arithmetic type, passed by value.
template <class Real>
struct DevParams {
  int n[3];            // cells per axis (n[2] = 1 in 2D)
  int bc[3];           // periodic / wall per axis
  int wall[3];         // obstacle rows at both ends of each axis
  int px;              // row pitch in elements (nx rounded up to 8)
  long long plane;     // elements between consecutive planes of a field
  Real eps;            // epsilon
  Real mob_eps;        // 1 / (tau_phi * eps)
  Real obst;           // 16 / (pi^2 eps)
  Real gamma[4][4], delta[4][4];
  Real inv2A[4];       // 1 / (2 A_a)
  Real inv4A[4];       // 1 / (4 A_a)
  Real chi_pure[4];    // 1 / inv2A[a], rounded as the device rounds 1 / chi (chi of a pure cell)
  Real ceq[4][2];
  Real S[4];
  Real dcl_ref[2];     // ceq_liquid - c_ref
  Real M0;             // D_liq / (2 A_liquid)
  Real at_eps;         // a_at * eps
  Real kappa0;         // 2 nu h / W0^2
  Real gbeta_c[2], gbeta_T;
  Real dT_ref;         // T_E - T_ref
  Real G;              // temperature gradient per cell
  Real inv_tau_f;      // 1 / tau_f
  Real force_pre;      // 1 - 1/(2 tau_f)
  Real q_floor;
  double theta0;       // -undercool - G v0: theta(v, t) = theta0 - G V t + G v
  double GV;           // G * V
  // appended last: earlier fields keep their parameter-bank offsets
  Real eta[4];         // shrinkage (rho_a - rho_0) / rho_0 per phase
  int shrink;          // 1 if any eta of the problem's phases is nonzero
  Real tilt_c[4][4];   // cos and sin of the turn of a pair's crystal axes about z
  Real tilt_s[4][4];
  int tilted;          // 1 if any pair of the problem's phases has a nonzero turn
  Real dceq_dT[4][2];  // ceq_a,i(T) = ceq[a][i] + dceq_dT[a][i] (T - T_E)
  int tdep;            // 1 if any of them is nonzero
  // 3D step over part of the vertical axis (a slab): the step advances the
  // planes v_lo .. v_hi - 1 of a grid of n[2] planes, and the field buffers
  // start at plane zbase.  A whole grid: v_lo = 0, v_hi = n[2], zbase = 0.
  int v_lo, v_hi, zbase;
  // 3D: tiles whose reach is pure liquid take the liquid path (per-tile
  // flags of the state); 0 = every tile takes the general path
  int liq_dispatch;
  // 1 if any pair of the problem's phases has a nonzero anisotropy delta, or
  // a turned crystal frame.  Otherwise dA/dq = 2 q, and a face flux needs
  // only the normal component of each face gradient (the transverse ones
  // are skipped, exactly).
  int aniso;
  // Byte offsets in a population buffer from a cell's population 0 (the
  // stored type's size): f_at[k] = k plane, the cell's own population k;
  // f_to[k] = f_at[k] + c_k . (1, px, px ny), where the collided population
  // k of a cell away from the edges lands.  Host-computed, so that each
  // access is one 64-bit add of a parameter to the cell's address.
  long long f_at[27], f_to[27];
};

// 1/x rounded to nearest: the same value as the IEEE division 1/x, by the
// correctly rounded reciprocal instead of the division routine.
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// Explicitly rounded operations: the compiler fuses a*b+c into one rounding
// where it sees fit, which may differ between two kernels; the arithmetic
// that the liquid path shares with the general path (in one kernel or two)
// is written with these so that both give the same bits.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

template <class Real>
__device__ __forceinline__ int fold_axis(const DevParams<Real>& P, int i, int a) {
  const int n = P.n[a];
  if (i < 0) i = P.bc[a] == kWall ? -1 - i : i + n;
  if (i >= n) i = P.bc[a] == kWall ? 2 * n - 1 - i : i - n;
  // tiles past a ragged end may reach further; those cells feed no output
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

template <class Real>
__device__ __forceinline__ bool obstacle(const DevParams<Real>& P, int x, int y, int z) {
  const int c[3] = {x, y, z};
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (P.wall[a] > 0 && (c[a] < P.wall[a] || c[a] >= P.n[a] - P.wall[a])) return true;
  return false;
}

// The element `off` bytes after p (population offsets f_at, f_to).
template <class T>
__device__ __forceinline__ T& at_bytes(T* p, long long off) {
  return *reinterpret_cast<T*>(reinterpret_cast<char*>(p) + off);
}
template <class T>
__device__ __forceinline__ const T& at_bytes(const T* p, long long off) {
  return *reinterpret_cast<const T*>(reinterpret_cast<const char*>(p) + off);
}

// ------------------------------------------------------------------ push streaming
// Where the populations of a cell stream to along one axis: the offset (in
// elements) of the +1 and -1 neighbour, periodic axes wrapping, and whether a
// wall lies in between (halfway bounce-back: a population that would cross
// it returns reversed into the cell itself).
struct PushAxis {
  int op, om;
  bool wp, wm;
};
__device__ __forceinline__ PushAxis push_axis(int i, int n, bool wall, int stride) {
  PushAxis a;
  a.wp = wall && i + 1 >= n;
  a.wm = wall && i - 1 < 0;
  a.op = (i + 1 < n ? 1 : (wall ? 0 : 1 - n)) * stride;
  a.om = (i - 1 >= 0 ? -1 : (wall ? 0 : n - 1)) * stride;
  return a;
}

// Stores population k of the cell at gi into its destination (one of the
// cells around it, or back into the cell reversed across a wall).
template <class Lat, class Store>
__device__ __forceinline__ void push_store(Store* __restrict__ f_out, long long plane, int gi, int k, Store v,
                                           const PushAxis& X, const PushAxis& Y, const PushAxis& Z) {
  constexpr int dims = Lat::D;
  const int c0 = Lat::c(k, 0), c1 = Lat::c(k, 1), c2 = dims == 3 ? Lat::c(k, 2) : 0;
  const bool bounce = (c0 > 0 && X.wp) || (c0 < 0 && X.wm) || (c1 > 0 && Y.wp) || (c1 < 0 && Y.wm) ||
                      (c2 > 0 && Z.wp) || (c2 < 0 && Z.wm);
  const int off = (c0 > 0 ? X.op : (c0 < 0 ? X.om : 0)) + (c1 > 0 ? Y.op : (c1 < 0 ? Y.om : 0)) +
                  (c2 > 0 ? Z.op : (c2 < 0 ? Z.om : 0));
  if (bounce)
    f_out[Lat::opp(k) * plane + gi] = v;
  else
    f_out[k * plane + gi + off] = v;
}

// ------------------------------------------------------------------ liquid tiles
// Liquid flags are kept per xy tile of the step grid and per plane: flag
// (tile, v) says that every cell the tile owns in plane v is pure liquid.
__device__ __forceinline__ long long liquid_flag_index(int bx, int by, int v, int gx, int gy) {
  return ((long long)v * gy + by) * gx + bx;
}

// The reach of the z segment starting at plane z0 of xy tile (bx, by) -- the
// 3 x 3 tiles around it (wrapped on periodic axes, skipped beyond walls,
// where a wall mirrors the tile's own cells) on planes z0 - 2 .. z0 + ZS + 1
// (folded like the cells) -- is flagged pure liquid.  Every thread of the CTA
// calls it; the answer is uniform.
template <int ZS, class Real>
__device__ __forceinline__ bool liquid_reach(const DevParams<Real>& P, const unsigned char* __restrict__ flags,
                                             int bx, int by, int z0, int gx, int gy) {
  __shared__ int s_all;
  if (threadIdx.x == 0) s_all = 1;
  __syncthreads();
  if (threadIdx.x < 9 * (ZS + 4)) {
    const int t = threadIdx.x % 9;
    const int v = fold_axis(P, z0 - 2 + (int)threadIdx.x / 9, 2);
    int c[2] = {bx + t % 3 - 1, by + t / 3 - 1};
    const int n[2] = {gx, gy};
    bool skip = false;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      if (c[a] < 0 || c[a] >= n[a]) {
        if (P.bc[a] == kWall) skip = true;
        c[a] = c[a] < 0 ? c[a] + n[a] : c[a] - n[a];
      }
    }
    if (!skip && !flags[liquid_flag_index(c[0], c[1], v, gx, gy)]) s_all = 0;
  }
  __syncthreads();
  return s_all != 0;
}

// ------------------------------------------------------------------ shared cell arithmetic
// Buoyancy drive of the melt at a cell: g beta_T (T - T_ref) +
// sum_i g beta_i (c_l,i(mu) - c_ref,i), theta = T - T_E; EXT: c_l,i at T.
template <int NC, bool EXT, class Real>
__device__ __forceinline__ Real buoyancy_drive(const DevParams<Real>& P, Real theta, const Real* mu) {
  Real drive = mul_rn(P.gbeta_T, add_rn(theta, P.dT_ref));
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    Real cl = P.dcl_ref[i];
    if constexpr (EXT) cl = fma_rn(P.dceq_dT[0][i], theta, cl);
    drive = fma_rn(P.gbeta_c[i], fma_rn(mu[i], P.inv2A[0], cl), drive);
  }
  return drive;
}

// Force-corrected velocity and total force of a cell (vertical axis D - 1):
// F_B = rho phl drive, U = (m + F_B/2) / (rho (1 + kappa/2)),
// F = F_B - rho kappa U, kappa = kappa0 (1 - phl)^2.
template <int D, class Real>
__device__ __forceinline__ void force_velocity(const DevParams<Real>& P, Real rho, Real phl, Real drive,
                                               const Real* m, Real* u, Real* F) {
  const Real sl = sub_rn(Real(1), phl);
  const Real kappa = mul_rn(mul_rn(P.kappa0, sl), sl);
  const Real FB = mul_rn(mul_rn(rho, phl), drive);
  const Real inv = rcp_rn(mul_rn(rho, fma_rn(Real(0.5), kappa, Real(1))));
  const Real rk = mul_rn(rho, kappa);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const Real fb = a == D - 1 ? FB : Real(0);
    u[a] = mul_rn(fma_rn(Real(0.5), fb, m[a]), inv);
    F[a] = fma_rn(-rk, u[a], fb);
  }
}

// Solute flux between two pure-liquid cells a, b (M = M0, h_l = 1):
// J = -M0 (mu_b - mu_a) + (u_a c_a + u_b c_b) / 2, c = ceq_l + mu / (2 A_l).
template <class Real>
__device__ __forceinline__ Real liquid_flux(const DevParams<Real>& P, Real ma, Real mb, Real ua, Real ub,
                                            Real ceqa, Real ceqb) {
  const Real adv = mul_rn(Real(0.5), fma_rn(ua, fma_rn(ma, P.inv2A[0], ceqa), mul_rn(ub, fma_rn(mb, P.inv2A[0], ceqb))));
  return fma_rn(-P.M0, sub_rn(mb, ma), adv);
}

// mu^{n+1} of an unchanged pure-liquid cell: mu + (-div - src) / (2 A_l)^-1.
template <class Real>
__device__ __forceinline__ Real liquid_mu(const DevParams<Real>& P, Real mu, Real div, Real src) {
  return fma_rn(sub_rn(-div, src), P.chi_pure[0], mu);
}

// ------------------------------------------------------------------ thermodynamics
// h_a(phi) = phi_a^2 (3 - 2 phi_a) + 2 phi_a sum_{b<g; b,g != a} phi_b phi_g
template <int NP, class Real>
__device__ __forceinline__ Real interp_h(const Real* p, int a) {
  Real s = Real(0);
#pragma unroll
  for (int b = 0; b < NP; ++b)
#pragma unroll
    for (int g = b + 1; g < NP; ++g)
      if (b != a && g != a) s += p[b] * p[g];
  return p[a] * p[a] * (Real(3) - Real(2) * p[a]) + Real(2) * p[a] * s;
}

// dh_b / dphi_a
template <int NP, class Real>
__device__ __forceinline__ Real interp_dh(const Real* p, int b, int a) {
  if (a == b) {
    Real s = Real(0);
#pragma unroll
    for (int g = 0; g < NP; ++g)
#pragma unroll
      for (int d = g + 1; d < NP; ++d)
        if (g != b && d != b) s += p[g] * p[d];
    return Real(6) * p[b] * (Real(1) - p[b]) + Real(2) * s;
  }
  Real s = Real(0);
#pragma unroll
  for (int d = 0; d < NP; ++d)
    if (d != a && d != b) s += p[d];
  return Real(2) * p[b] * s;
}

// dA/dq_j for A(q) = ac(q)^2 |q|^2, ac = 1 - delta (3 - 4 sum q^4 / |q|^4).
// Only component j is returned, but it depends on all of q.
template <int D, class Real>
__device__ __forceinline__ Real dAdq(const Real* q, Real delta, Real q_floor, int j) {
  if (delta == Real(0)) return Real(2) * q[j];  // isotropic pair
  Real s2 = Real(0), s4 = Real(0);
#pragma unroll
  for (int t = 0; t < D; ++t) {
    s2 += q[t] * q[t];
    s4 += q[t] * q[t] * q[t] * q[t];
  }
  if (s2 <= q_floor) return Real(2) * q[j];
  const Real inv2 = Real(1) / s2;
  const Real r4 = s4 * inv2 * inv2;
  const Real ac = Real(1) - delta * (Real(3) - Real(4) * r4);
  const Real qj = q[j];
  const Real dac = Real(16) * delta * (qj * qj * qj - qj * s4 * inv2) * inv2 * inv2;
  return Real(2) * ac * (ac * qj + s2 * dac);
}

// BGK collision with Guo forcing, in deviations: for every k,
//   f*_k - w_k = omega d_k + w_k [alpha + c_k.v + (c_k.U)(c_k.z)],
//   alpha = (drho - 1.5 rho U.U) / tau - 3 pre U.F,
//   v = 3 (rho U / tau + pre F),  z = 4.5 rho U / tau + 9 pre F,
// with omega = 1 - 1/tau and pre = 1 - 1/(2 tau): the second-order
// equilibrium over tau plus the discrete force, collected by powers of c_k.
// Opposite directions share alpha and the quadratic term and flip the linear
// one, so each pair costs one evaluation.  put(k, value) stores a result.
template <int Q, class Real, class Put>
__device__ __forceinline__ void collide(const DevParams<Real>& P, const Real* dk, Real drho, Real rho,
                                        const Real* u, const Real* F, Put&& put) {
  using Lat = Lattice<Q>;
  constexpr int D = Lat::D;
  const Real itau = P.inv_tau_f, pre = P.force_pre, omega = Real(1) - itau;
  // every product and sum rounded as written (fma_rn etc.), so that the two
  // 3D kernels, which both collide liquid cells, give the same bits
  const Real irho = mul_rn(itau, rho), pre9 = mul_rn(Real(9), pre);
  Real uu = Real(0), uF = Real(0), v[D], z[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    uu = fma_rn(u[a], u[a], uu);
    uF = fma_rn(u[a], F[a], uF);
    const Real ru = mul_rn(irho, u[a]);
    v[a] = mul_rn(Real(3), fma_rn(pre, F[a], ru));
    z[a] = fma_rn(Real(4.5), ru, mul_rn(pre9, F[a]));
  }
  const Real alpha =
      fma_rn(itau, fma_rn(mul_rn(Real(-1.5), rho), uu, drho), mul_rn(mul_rn(Real(-3), pre), uF));
  put(0, fma_rn(omega, dk[0], mul_rn(Real(Lat::w(0)), alpha)));
#pragma unroll
  for (int k = 1; k < Q; ++k) {
    if (Lat::opp(k) < k) continue;  // each pair once, at its first index
    const int kb = Lat::opp(k);
    Real cu = Real(0), cz = Real(0), cv = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if (Lat::c(k, a) > 0) {
        cu += u[a];
        cz += z[a];
        cv += v[a];
      } else if (Lat::c(k, a) < 0) {
        cu -= u[a];
        cz -= z[a];
        cv -= v[a];
      }
    }
    const Real wk = Real(Lat::w(k));
    const Real wq = mul_rn(wk, fma_rn(cu, cz, alpha)), wl = mul_rn(wk, cv);
    put(k, fma_rn(omega, dk[k], add_rn(wq, wl)));
    put(kb, fma_rn(omega, dk[kb], sub_rn(wq, wl)));
  }
}

// Full vector dA/dq (for the centre term).
template <int D, class Real>
__device__ __forceinline__ void dAdq_vec(const Real* q, Real delta, Real q_floor, Real* out) {
  Real s2 = Real(0), s4 = Real(0);
  if (delta != Real(0)) {  // an isotropic pair needs neither sum
#pragma unroll
    for (int t = 0; t < D; ++t) {
      s2 += q[t] * q[t];
      s4 += q[t] * q[t] * q[t] * q[t];
    }
  }
  if (delta == Real(0) || s2 <= q_floor) {
#pragma unroll
    for (int t = 0; t < D; ++t) out[t] = Real(2) * q[t];
    return;
  }
  const Real inv2 = Real(1) / s2;
  const Real r4 = s4 * inv2 * inv2;
  const Real ac = Real(1) - delta * (Real(3) - Real(4) * r4);
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const Real qt = q[t];
    const Real dac = Real(16) * delta * (qt * qt * qt - qt * s4 * inv2) * inv2 * inv2;
    out[t] = Real(2) * ac * (ac * qt + s2 * dac);
  }
}

// dA/dq_j of pair (a, b).  With TILT its crystal axes are turned by theta
// about z: the cubic anisotropy is a function of the crystal-frame
// components r = (c q_x + s q_y, -s q_x + c q_y, q_z) and, by the chain rule,
// dA/dq = (c r'_x - s r'_y, s r'_x + c r'_y, r'_z) with r' = dA/dr.
template <int D, bool TILT, class Real>
__device__ __forceinline__ Real dAdq_pair(const DevParams<Real>& P, int a, int b, const Real* q, int j) {
  if constexpr (!TILT) {
    return dAdq<D>(q, P.delta[a][b], P.q_floor, j);
  } else {
    const Real c = P.tilt_c[a][b], s = P.tilt_s[a][b];
    Real r[D];
    r[0] = c * q[0] + s * q[1];
    r[1] = c * q[1] - s * q[0];
    if constexpr (D == 3) r[2] = q[2];
    if (j == 2) return dAdq<D>(r, P.delta[a][b], P.q_floor, 2);
    const Real d0 = dAdq<D>(r, P.delta[a][b], P.q_floor, 0);
    const Real d1 = dAdq<D>(r, P.delta[a][b], P.q_floor, 1);
    return j == 0 ? c * d0 - s * d1 : s * d0 + c * d1;
  }
}

// Full vector dA/dq of pair (a, b), turned as dAdq_pair.
template <int D, bool TILT, class Real>
__device__ __forceinline__ void dAdq_vec_pair(const DevParams<Real>& P, int a, int b, const Real* q,
                                              Real* out) {
  if constexpr (!TILT) {
    dAdq_vec<D>(q, P.delta[a][b], P.q_floor, out);
  } else {
    const Real c = P.tilt_c[a][b], s = P.tilt_s[a][b];
    Real r[D], d[D];
    r[0] = c * q[0] + s * q[1];
    r[1] = c * q[1] - s * q[0];
    if constexpr (D == 3) r[2] = q[2];
    dAdq_vec<D>(r, P.delta[a][b], P.q_floor, d);
    out[0] = c * d[0] - s * d[1];
    out[1] = s * d[0] + c * d[1];
    if constexpr (D == 3) out[2] = d[2];
  }
}

// Euclidean projection of the m active values onto {sum = 1, u >= 0}
// (sort and threshold; m <= 4).
template <class Real, int NMAX>
__device__ __forceinline__ void project_simplex(Real* u, int m) {
  Real s[NMAX];
#pragma unroll
  for (int j = 0; j < NMAX; ++j) s[j] = j < m ? u[j] : Real(-1e30);
#pragma unroll
  for (int i = 0; i < NMAX; ++i)
#pragma unroll
    for (int j = 0; j + 1 < NMAX - i; ++j)
      if (s[j] < s[j + 1]) {
        Real t = s[j];
        s[j] = s[j + 1];
        s[j + 1] = t;
      }
  Real run = Real(0), theta = Real(0);
#pragma unroll
  for (int j = 0; j < NMAX; ++j) {
    if (j < m) {
      run += s[j];
      const Real t = (run - Real(1)) / Real(j + 1);
      if (s[j] - t > Real(0)) theta = t;
    }
  }
#pragma unroll
  for (int j = 0; j < NMAX; ++j)
    if (j < m) u[j] = u[j] - theta > Real(0) ? u[j] - theta : Real(0);
}

// ------------------------------------------------------------------ phase field
// Stored planes: N = 2 keeps only phi_1 (phi_0 = 1 - phi_1); N >= 3 keeps
// all N planes.
template <int NP>
struct PhiStore {
  static constexpr int NS = NP == 2 ? 1 : NP;
};

// The phase at exactly 1 when every other phase is exactly 0 (its h is then
// the unit vector of that phase, exactly), else -1.
template <int NP, class Real>
__device__ __forceinline__ int pure_phase(const Real* v) {
  int pa = -1, n1 = 0, n0 = 0;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    if (v[a] == Real(1)) {
      pa = a;
      ++n1;
    } else if (v[a] == Real(0)) {
      ++n0;
    }
  }
  return (n1 == 1 && n0 == NP - 1) ? pa : -1;
}

template <int NP, class Real, class Index>
__device__ __forceinline__ void load_phases(const Real* __restrict__ phi, Index g,
                                            long long plane, Real* v) {
  if (NP == 2) {
    v[1] = phi[g];
    v[0] = Real(1) - v[1];
  } else {
#pragma unroll
    for (int a = 0; a < NP; ++a) v[a] = (phi + a * plane)[g];
  }
}

template <int D, class Real>
__device__ __forceinline__ long long cell_index(const DevParams<Real>& P, int x, int y, int z) {
  return (long long)x + (long long)P.px * ((long long)y + (long long)P.n[1] * z);
}

// ------------------------------------------------------------------ state I/O
// Moving frame: layer v of every plane of dst takes layer
// min(v + rows, nv - 1) of src.  W is a word of the stored type's size; the
// layout is the padded one (`layer` words per vertical layer, `n` words per
// plane in use, planes `plane` words apart).  dst and src do not overlap.
template <class W>
__global__ void shift_frame_kernel(const W* __restrict__ src, W* __restrict__ dst, int planes,
                                   long long plane, long long n, long long layer, int nv, int rows) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int v = (int)(i / layer);
  const long long j = i + (long long)(min(v + rows, nv - 1) - v) * layer;
  for (int p = 0; p < planes; ++p) dst[p * plane + i] = src[p * plane + j];
}

// phi from N exchange planes (liquid first) to the stored planes.
// Offset of logical cell x (x fastest, no padding) in the padded layout.
__device__ __forceinline__ long long padded(long long x, int nx, int px) {
  return (x % nx) + (long long)px * (x / nx);
}

template <int NP, class Real, class In>
__global__ void load_phi_kernel(long long cells, int nx, int px, long long plane,
                                const In* __restrict__ src, Real* __restrict__ dst) {
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (x >= cells) return;
  const long long o = padded(x, nx, px);
  if (NP == 2) {
    dst[o] = Real(src[cells + x]);
  } else {
#pragma unroll
    for (int a = 0; a < NP; ++a) dst[a * plane + o] = Real(src[a * cells + x]);
  }
}

template <int NC, class Real, class In>
__global__ void load_mu_kernel(long long cells, int nx, int px, long long plane,
                               const In* __restrict__ src, Real* __restrict__ dst) {
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (x >= cells) return;
  const long long o = padded(x, nx, px);
#pragma unroll
  for (int i = 0; i < NC; ++i) dst[i * plane + o] = Real(src[i * cells + x]);
}

// f (full populations, or the fluid at rest when src is null) to deviations.
template <int Q, class Store, class In>
__global__ void load_f_kernel(long long cells, int nx, int px, long long plane,
                              const In* __restrict__ src, Store* __restrict__ dst) {
  using Lat = Lattice<Q>;
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (x >= cells) return;
  const long long o = padded(x, nx, px);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    using R = typename std::conditional<std::is_same<Store, double>::value, double, float>::type;
    const R d = src ? R(src[k * cells + x]) - R(Lat::w(k)) : R(0);
    dst[k * plane + o] = Codec<Store>::put(d);
  }
}

// V consecutive words as one access of V * sizeof(T) bytes (2, 4, 8 or 16),
// at an address aligned to that size.
template <int B>
struct Bytes;
template <>
struct Bytes<2> { using type = unsigned short; };
template <>
struct Bytes<4> { using type = unsigned; };
template <>
struct Bytes<8> { using type = uint2; };
template <>
struct Bytes<16> { using type = uint4; };

template <int V, class T>
__device__ __forceinline__ void load_words(const T* __restrict__ p, T (&v)[V]) {
  using W = typename Bytes<V * (int)sizeof(T)>::type;
  const W w = *reinterpret_cast<const W*>(p);
  memcpy(v, &w, sizeof(W));
}

template <int V, class T>
__device__ __forceinline__ void store_words(T* __restrict__ p, const T (&v)[V]) {
  using W = typename Bytes<V * (int)sizeof(T)>::type;
  W w;
  memcpy(&w, v, sizeof(W));
  *reinterpret_cast<W*>(p) = w;
}

// The whole of S^n from exchange planes in one launch: phi (N planes, liquid
// first; the stored planes), mu (K-1 planes), f (Q planes of populations, or
// the fluid at rest when src_f is null) as deviations, the step counter of
// the loaded buffer (clock_a) and of the other one (clock_b, when not null).
// Each thread takes V consecutive cells of a
// row (nx a multiple of V and, for V > 1, the sources 16-byte aligned), and
// issues every load of its cells before the first store, so that the reads
// of a host source over the host link are all in flight together.  The
// arithmetic is that of load_phi_kernel, load_mu_kernel and load_f_kernel.
template <int NP, int NC, int Q, class Real, class Store, int V>
__global__ void load_state_kernel(long long cells, int nx, int px, long long plane,
                                  const Real* __restrict__ src_phi, const Real* __restrict__ src_mu,
                                  const Real* __restrict__ src_f, Real* __restrict__ phi,
                                  Real* __restrict__ mu, Store* __restrict__ f,
                                  double* __restrict__ clock_a, double* __restrict__ clock_b,
                                  double t0) {
  using Lat = Lattice<Q>;
  using R = typename std::conditional<std::is_same<Store, double>::value, double, float>::type;
  constexpr int NS = PhiStore<NP>::NS;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clock_a[0] = t0;
    if (clock_b) clock_b[0] = t0;
  }
  // a grid-stride loop: the launcher caps the grid (two CTAs per SM), so
  // that a load and a field write-back over the host link can share the SMs
  const long long stride = (long long)gridDim.x * blockDim.x * V;
  for (long long x = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * V; x < cells; x += stride) {
    const long long o = padded(x, nx, px);
    Real vp[NS][V], vm[NC][V], vf[Q][V];
#pragma unroll
    for (int s = 0; s < NS; ++s) load_words<V>(src_phi + (NP == 2 ? 1 : s) * cells + x, vp[s]);
#pragma unroll
    for (int i = 0; i < NC; ++i) load_words<V>(src_mu + i * cells + x, vm[i]);
    if (src_f) {
#pragma unroll
      for (int k = 0; k < Q; ++k) load_words<V>(src_f + k * cells + x, vf[k]);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) store_words<V>(phi + s * plane + o, vp[s]);
#pragma unroll
    for (int i = 0; i < NC; ++i) store_words<V>(mu + i * plane + o, vm[i]);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      Store d[V];
#pragma unroll
      for (int j = 0; j < V; ++j) d[j] = Codec<Store>::put(src_f ? R(vf[k][j]) - R(Lat::w(k)) : R(0));
      store_words<V>(f + k * plane + o, d);
    }
  }
}

// Exchange-format fields of the current state; any output may be null.
// phi: N planes (liquid first); c_i = sum_a h_a (ceq_a,i(T) + mu_i / (2 A_a));
// f = w + d; rho = 1 + sum d; U as in the step (force-corrected); dev = d.
template <int D, int Q, int NP, int NC, class Real, class Store, class Out>
__device__ __forceinline__ void fields_cell(const DevParams<Real>& P, const Real* __restrict__ phi,
                                            const Real* __restrict__ mu_in, const Store* __restrict__ f,
                                            const double* __restrict__ clock, Out* __restrict__ o_phi,
                                            Out* __restrict__ o_mu, Out* __restrict__ o_c,
                                            Out* __restrict__ o_f, Out* __restrict__ o_rho,
                                            Out* __restrict__ o_u, Out* __restrict__ o_dev,
                                            long long cells, long long x) {
  using Lat = Lattice<Q>;
  const int gx = (int)(x % P.n[0]);
  const int gy = (int)((x / P.n[0]) % P.n[1]);
  const int gz = (int)(x / ((long long)P.n[0] * P.n[1]));
  const long long o = cell_index<D>(P, gx, gy, gz);
  Real p[NP], mu[NC];
  load_phases<NP>(phi, o, P.plane, p);
#pragma unroll
  for (int i = 0; i < NC; ++i) mu[i] = mu_in[i * P.plane + o];
  if (o_phi)
#pragma unroll
    for (int a = 0; a < NP; ++a) o_phi[a * cells + x] = Out(p[a]);
  if (o_mu)
#pragma unroll
    for (int i = 0; i < NC; ++i) o_mu[i * cells + x] = Out(mu[i]);
  const int v_coord = D == 3 ? gz : gy;
  const Real theta = Real(P.theta0 - P.GV * clock[0]) + P.G * Real(v_coord);  // T - T_E
  if (o_c) {
    Real h[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) h[a] = interp_h<NP>(p, a);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      Real c = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) c += h[a] * (P.ceq[a][i] + P.dceq_dT[a][i] * theta + mu[i] * P.inv2A[a]);
      o_c[i * cells + x] = Out(c);
    }
  }
  // the populations only where an output needs them (uniform across the grid)
  if (!o_f && !o_dev && !o_rho && !o_u) return;
  Real drho = Real(0), m[D];
#pragma unroll
  for (int a = 0; a < D; ++a) m[a] = Real(0);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const Real dk = Codec<Store>::load(f[k * P.plane + o]);
    drho += dk;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (Lat::c(k, a) != 0) m[a] += Real(Lat::c(k, a)) * dk;
    if (o_f) o_f[k * cells + x] = Out(Real(Lat::w(k)) + dk);
    if (o_dev) o_dev[k * cells + x] = Out(dk);
  }
  const Real rho = Real(1) + drho;
  if (o_rho) o_rho[x] = Out(rho);
  if (o_u) {
    const Real phil = obstacle(P, gx, gy, gz) ? Real(0) : p[0];
    const Real sl = Real(1) - phil;
    const Real kappa = P.kappa0 * sl * sl;
    Real drive = P.gbeta_T * (theta + P.dT_ref);
#pragma unroll
    for (int i = 0; i < NC; ++i)
      drive += P.gbeta_c[i] * (P.dcl_ref[i] + P.dceq_dT[0][i] * theta + mu[i] * P.inv2A[0]);
    const Real FB = rho * phil * drive;
    const Real inv = rcp_rn(rho * (Real(1) + Real(0.5) * kappa));
#pragma unroll
    for (int a = 0; a < D; ++a) o_u[a * cells + x] = Out((m[a] + (a == D - 1 ? Real(0.5) * FB : Real(0))) * inv);
  }
}

// One thread per cell, in a grid-stride loop over a grid the launcher caps
// at two CTAs per SM (see load_state_kernel).
template <int D, int Q, int NP, int NC, class Real, class Store, class Out>
__global__ void fields_kernel(const DevParams<Real> P, const Real* __restrict__ phi,
                              const Real* __restrict__ mu_in, const Store* __restrict__ f,
                              const double* __restrict__ clock, Out* __restrict__ o_phi,
                              Out* __restrict__ o_mu, Out* __restrict__ o_c, Out* __restrict__ o_f,
                              Out* __restrict__ o_rho, Out* __restrict__ o_u,
                              Out* __restrict__ o_dev) {
  const long long cells = (long long)P.n[0] * P.n[1] * P.n[2];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < cells; x += stride)
    fields_cell<D, Q, NP, NC, Real, Store, Out>(P, phi, mu_in, f, clock, o_phi, o_mu, o_c, o_f,
                                                o_rho, o_u, o_dev, cells, x);
}

// ------------------------------------------------------------------ invariants
// Per-cell totals in FP64 without fused multiply-add, in a fixed order, and
// a fixed-order block reduction (see gpflbm_invariants in gpflbm.h).
struct InvParams {
  long long cells, plane;
  int nx, px;
  double ceq[4][2];
  double inv2A[4];
  // temperature-dependent ceq: T - T_E = theta_t + G v, v = x / vlayer
  double dceq_dT[4][2];
  double theta_t, G;
  long long vlayer;
  int tdep;
};

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 608;

template <int NP>
__device__ __forceinline__ double h_exact(const double* p, int a) {
  double s = 0.0;
#pragma unroll
  for (int b = 0; b < NP; ++b)
#pragma unroll
    for (int g = b + 1; g < NP; ++g)
      if (b != a && g != a) s = __dadd_rn(s, __dmul_rn(p[b], p[g]));
  const double t1 = __dmul_rn(__dmul_rn(p[a], p[a]), __dsub_rn(3.0, __dmul_rn(2.0, p[a])));
  const double t2 = __dmul_rn(__dmul_rn(2.0, p[a]), s);
  return __dadd_rn(t1, t2);
}

__device__ __forceinline__ double warp_sum_butterfly(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// out[b * (NC + 3) + j]: j = 0 mass deviation, 1..NC solutes, NC+1 solid,
// NC+2 count of non-finite cells (as a double).
template <int Q, int NP, int NC, class Real, class Store>
__global__ void __launch_bounds__(kRedThreads)
    invariants_kernel(const InvParams P, const Real* __restrict__ phi, const Real* __restrict__ mu,
                      const Store* __restrict__ f, double* __restrict__ partial) {
  constexpr int NV = NC + 3;
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  const long long stride = (long long)gridDim.x * kRedThreads;
  for (long long x = blockIdx.x * (long long)kRedThreads + threadIdx.x; x < P.cells; x += stride) {
    const long long o = padded(x, P.nx, P.px);
    double p[NP], m[NC];
    if (NP == 2) {
      p[1] = (double)phi[o];
      p[0] = __dsub_rn(1.0, p[1]);
    } else {
#pragma unroll
      for (int a = 0; a < NP; ++a) p[a] = (double)phi[a * P.plane + o];
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) m[i] = (double)mu[i * P.plane + o];
    double dm = 0.0;
#pragma unroll
    for (int k = 0; k < Q; ++k) dm = __dadd_rn(dm, (double)Codec<Store>::load(f[k * P.plane + o]));
    double h[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) h[a] = h_exact<NP>(p, a);
    double v[NV];
    v[0] = dm;
    const double th = P.tdep ? __dadd_rn(P.theta_t, __dmul_rn(P.G, (double)(x / P.vlayer))) : 0.0;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      double c = 0.0;
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        const double ce = P.tdep ? __dadd_rn(P.ceq[a][i], __dmul_rn(P.dceq_dT[a][i], th)) : P.ceq[a][i];
        c = __dadd_rn(c, __dmul_rn(h[a], __dadd_rn(ce, __dmul_rn(m[i], P.inv2A[a]))));
      }
      v[1 + i] = c;
    }
    double sol = 0.0;
#pragma unroll
    for (int a = 1; a < NP; ++a) sol = __dadd_rn(sol, h[a]);
    v[NC + 1] = sol;
    bool finite = isfinite(dm);
#pragma unroll
    for (int a = 0; a < NP; ++a) finite = finite && isfinite(p[a]);
#pragma unroll
    for (int i = 0; i < NC; ++i) finite = finite && isfinite(m[i]);
    v[NC + 2] = finite ? 0.0 : 1.0;
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = __dadd_rn(acc[j], v[j]);
  }
  __shared__ double s_w[kRedThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const double w = warp_sum_butterfly(acc[j]);
    if (lane == 0) s_w[warp][j] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = s_w[0][j];
      for (int w = 1; w < kRedThreads / 32; ++w) s = __dadd_rn(s, s_w[w][j]);
      partial[blockIdx.x * NV + j] = s;
    }
  }
}

// Adds the block partials in block order (one thread).
template <int NV>
__global__ void invariants_finish_kernel(const double* __restrict__ partial, int blocks,
                                         double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = 0; j < NV; ++j) {
    double s = partial[j];
    for (int b = 1; b < blocks; ++b) s = __dadd_rn(s, partial[b * NV + j]);
    out[j] = s;
  }
}

}  // namespace gpflbm

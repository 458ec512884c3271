// Device code of the coupled Grand-Potential phase-field / lattice-Boltzmann
// step for sm_103a.  Two kernels per time step, in the order of Algorithm 1:
//
//   phase_field_kernel  : phi^n, mu^n            -> phi^{n+1}       (Eq. PhfGrand)
//   mu_lbm_kernel       : phi^n, phi^{n+1}, mu^n, f^n -> mu^{n+1}, f^{n+1}
//                         (Eq. conc in flux form; Eq. LBMEq_1 with Eq. f^eq,
//                          Eq. discreteForce, drag G_D, buoyancy G_B, Eq. rhovel)
//
// Both kernels stage their inputs for a tile plus a one-cell halo in shared
// memory, evaluate every face flux of the tile once (a face is shared by two
// cells), and write one cell per thread.  Populations are kept as the
// deviation d_k = f_k - w_k so that FP32 keeps the small momentum
// m = sum_k c_k d_k to full relative precision; with 16-bit storage the
// deviation is the stored quantity.  No tensor cores: the step is a
// bandwidth-bound stencil.
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

template <int D>
struct LatticeOf;
template <>
struct LatticeOf<2> {
  using type = Lattice<9>;
};
template <>
struct LatticeOf<3> {
  using type = Lattice<19>;
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

// ------------------------------------------------------------------ tiles
template <int D, class Real>
struct Tile;
template <>
struct Tile<2, float> {
  static constexpr int TX = 64, TY = 8, TZ = 1;
};
template <>
struct Tile<2, double> {
  static constexpr int TX = 32, TY = 8, TZ = 1;
};
template <>
struct Tile<3, float> {
  static constexpr int TX = 32, TY = 4, TZ = 2;
};
template <>
struct Tile<3, double> {
  static constexpr int TX = 16, TY = 4, TZ = 2;
};

template <int D, class Real>
struct Geo {
  static constexpr int TX = Tile<D, Real>::TX, TY = Tile<D, Real>::TY, TZ = Tile<D, Real>::TZ;
  static constexpr int NT = TX * TY * TZ;
  // halo box: one cell on each side (no z halo in 2D)
  static constexpr int HX = TX + 2, HY = TY + 2, HZ = D == 3 ? TZ + 2 : 1;
  static constexpr int HC = HX * HY * HZ;
  static constexpr int SX = 1, SY = HX, SZ = HX * HY;  // halo strides
  static constexpr int ZOFF = D == 3 ? 1 : 0;          // halo offset along z
  // faces normal to each axis: the lower face of every tile cell plus the
  // upper face of the last cell
  static constexpr int F0 = (TX + 1) * TY * TZ;
  static constexpr int F1 = TX * (TY + 1) * TZ;
  static constexpr int F2 = D == 3 ? TX * TY * (TZ + 1) : 0;
  static constexpr int FALL = F0 + F1 + F2;
  __host__ __device__ static constexpr int hstride(int a) { return a == 0 ? SX : (a == 1 ? SY : SZ); }
  __host__ __device__ static constexpr int fcount(int a) { return a == 0 ? F0 : (a == 1 ? F1 : F2); }
  __host__ __device__ static constexpr int foff(int a) { return a == 0 ? 0 : (a == 1 ? F0 : F0 + F1); }
  // face grid extent along axis b for faces normal to axis a
  __host__ __device__ static constexpr int fext(int a, int b) {
    return (b == 0 ? TX : (b == 1 ? TY : TZ)) + (a == b ? 1 : 0);
  }
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
};

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
  Real s2 = Real(0), s4 = Real(0);
#pragma unroll
  for (int t = 0; t < D; ++t) {
    s2 += q[t] * q[t];
    s4 += q[t] * q[t] * q[t] * q[t];
  }
  if (delta == Real(0) || s2 <= q_floor) return Real(2) * q[j];
  const Real inv2 = Real(1) / s2;
  const Real r4 = s4 * inv2 * inv2;
  const Real ac = Real(1) - delta * (Real(3) - Real(4) * r4);
  const Real qj = q[j];
  const Real dac = Real(16) * delta * (qj * qj * qj - qj * s4 * inv2) * inv2 * inv2;
  return Real(2) * ac * (ac * qj + s2 * dac);
}

// Full vector dA/dq (for the centre term).
template <int D, class Real>
__device__ __forceinline__ void dAdq_vec(const Real* q, Real delta, Real q_floor, Real* out) {
  Real s2 = Real(0), s4 = Real(0);
#pragma unroll
  for (int t = 0; t < D; ++t) {
    s2 += q[t] * q[t];
    s4 += q[t] * q[t] * q[t] * q[t];
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

template <int NP, class Real>
__device__ __forceinline__ void load_phases(const Real* __restrict__ phi, long long g,
                                            long long plane, Real* v) {
  if (NP == 2) {
    v[1] = phi[g];
    v[0] = Real(1) - v[1];
  } else {
#pragma unroll
    for (int a = 0; a < NP; ++a) v[a] = phi[a * plane + g];
  }
}

template <int D, class Real>
__device__ __forceinline__ long long cell_index(const DevParams<Real>& P, int x, int y, int z) {
  return (long long)x + (long long)P.px * ((long long)y + (long long)P.n[1] * z);
}

// True when the tile and its one-cell halo lie inside the domain on every
// axis, so halo cells need no wrapping or mirroring (block-uniform).
template <int D, class Real>
__device__ __forceinline__ bool tile_inside(const DevParams<Real>& P, const int* b0) {
  using G = Geo<D, Real>;
  const int T[3] = {G::TX, G::TY, G::TZ};
  bool in = true;
#pragma unroll
  for (int a = 0; a < D; ++a) in = in && b0[a] >= 1 && b0[a] + T[a] + 1 <= P.n[a];
  return in;
}

// Global coordinates of halo cell h of the tile at b0 (halo offset 1 per axis).
template <int D, class Real>
__device__ __forceinline__ void halo_coords(const DevParams<Real>& P, const int* b0, bool inner,
                                            int h, int* c) {
  using G = Geo<D, Real>;
  const int hx = h % G::HX, hy = (h / G::HX) % G::HY, hz = h / (G::HX * G::HY);
  if (inner) {
    c[0] = b0[0] + hx - 1;
    c[1] = b0[1] + hy - 1;
    c[2] = D == 3 ? b0[2] + hz - 1 : 0;
  } else {
    c[0] = fold_axis(P, b0[0] + hx - 1, 0);
    c[1] = fold_axis(P, b0[1] + hy - 1, 1);
    c[2] = D == 3 ? fold_axis(P, b0[2] + hz - 1, 2) : 0;
  }
}

// Shared-memory layout of the phase-field kernel (bytes).
template <int D, int NP, class Real>
struct PfSmem {
  using G = Geo<D, Real>;
  static constexpr size_t phi = 0;
  static constexpr size_t flux = phi + sizeof(Real) * NP * G::HC;
  static constexpr size_t mask = flux + sizeof(Real) * NP * G::FALL;
  static constexpr size_t multi = mask + G::HC;
  static constexpr size_t bytes = multi + G::NT + 16;
};

template <int D, int NP, int NC, class Real>
__global__ void __launch_bounds__(Geo<D, Real>::NT)
    phase_field_kernel(const DevParams<Real> P, const Real* __restrict__ phi_in,
                       const Real* __restrict__ mu_in, Real* __restrict__ phi_out,
                       const double* __restrict__ clock) {
  using G = Geo<D, Real>;
  using L = PfSmem<D, NP, Real>;
  constexpr int NS = PhiStore<NP>::NS;
  extern __shared__ __align__(16) unsigned char smem[];
  Real* s_phi = reinterpret_cast<Real*>(smem + L::phi);
  Real* s_flux = reinterpret_cast<Real*>(smem + L::flux);
  unsigned char* s_mask = smem + L::mask;
  unsigned char* s_multi = smem + L::multi;

  const int tid = threadIdx.x;
  const int b0[3] = {(int)blockIdx.x * G::TX, (int)blockIdx.y * G::TY, (int)blockIdx.z * G::TZ};
  const bool inner = tile_inside<D>(P, b0);

  // 1. phi^n on the tile and its halo, plus the set of phases present
  for (int h = tid; h < G::HC; h += G::NT) {
    int c[3];
    halo_coords<D>(P, b0, inner, h, c);
    Real v[NP];
    load_phases<NP>(phi_in, cell_index<D>(P, c[0], c[1], c[2]), P.plane, v);
    unsigned m = 0;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      s_phi[a * G::HC + h] = v[a];
      if (v[a] > Real(0)) m |= 1u << a;
    }
    s_mask[h] = (unsigned char)m;
  }
  __syncthreads();

  // 2. cells with more than one phase in their 3^d neighbourhood; elsewhere
  //    the single present phase keeps phi = 1 (its rate g - Lambda is 0)
  const int t3[3] = {tid % G::TX, (tid / G::TX) % G::TY, tid / (G::TX * G::TY)};
  const int gx = b0[0] + t3[0], gy = b0[1] + t3[1], gz = b0[2] + t3[2];
  const bool inside = gx < P.n[0] && gy < P.n[1] && gz < P.n[2];
  const int h = (t3[0] + 1) * G::SX + (t3[1] + 1) * G::SY + (t3[2] + G::ZOFF) * G::SZ;
  unsigned act = 0;
#pragma unroll
  for (int dz = -(D == 3 ? 1 : 0); dz <= (D == 3 ? 1 : 0); ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) act |= s_mask[h + dx * G::SX + dy * G::SY + dz * G::SZ];
  const bool multi = inside && __popc(act) >= 2 && !obstacle(P, gx, gy, gz);
  s_multi[tid] = multi ? 1 : 0;
  const long long g = inside ? cell_index<D>(P, gx, gy, gz) : 0;
  if (!__syncthreads_or(multi)) {
    if (inside)
#pragma unroll
      for (int s = 0; s < NS; ++s) phi_out[s * P.plane + g] = s_phi[(NP == 2 ? 1 : s) * G::HC + h];
    return;
  }

  // 3. d-th component of da/d(grad phi_a) on the faces of multi-phase cells:
  //    -sum_{b != a} gamma_ab phi_b dA/dq(q_ab), q_ab = phi_a grad phi_b - phi_b grad phi_a
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int ex = G::fext(d, 0), ey = G::fext(d, 1);
    const int tstride = d == 0 ? 1 : (d == 1 ? G::TX : G::TX * G::TY);
    const int Td = d == 0 ? G::TX : (d == 1 ? G::TY : G::TZ);
    for (int i = tid; i < G::fcount(d); i += G::NT) {
      const int f[3] = {i % ex, (i / ex) % ey, i / (ex * ey)};
      const int tu = f[0] + G::TX * (f[1] + G::TY * f[2]);  // upper tile cell (if f[d] < Td)
      const bool need = (f[d] < Td && s_multi[tu]) || (f[d] > 0 && s_multi[tu - tstride]);
      const int gd = b0[d] + f[d];  // global index of the upper cell of the face
      const bool closed = P.bc[d] == kWall && (gd == 0 || gd == P.n[d]);
      Real fl[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) fl[a] = Real(0);
      if (need && !closed) {
        const int hb = (f[0] + 1) * G::SX + (f[1] + 1) * G::SY + (f[2] + G::ZOFF) * G::SZ;
        const int ha = hb - G::hstride(d);
        Real pf[NP], gr[NP][D];
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          const Real* sp = s_phi + a * G::HC;
          pf[a] = Real(0.5) * (sp[ha] + sp[hb]);
#pragma unroll
          for (int t = 0; t < D; ++t) {
            if (t == d) {
              gr[a][t] = sp[hb] - sp[ha];
            } else {
              const int st = G::hstride(t);
              gr[a][t] = Real(0.25) * (sp[ha + st] + sp[hb + st] - sp[ha - st] - sp[hb - st]);
            }
          }
        }
#pragma unroll
        for (int a = 0; a < NP; ++a)
#pragma unroll
          for (int b = a + 1; b < NP; ++b) {
            const Real gab = P.gamma[a][b];
            if (gab == Real(0)) continue;
            Real q[D];
#pragma unroll
            for (int t = 0; t < D; ++t) q[t] = pf[a] * gr[b][t] - pf[b] * gr[a][t];
            const Real v = dAdq<D>(q, P.delta[a][b], P.q_floor, d);
            fl[a] -= gab * pf[b] * v;  // dA/dq(q_ba) = -dA/dq(q_ab)
            fl[b] += gab * pf[a] * v;
          }
      }
#pragma unroll
      for (int a = 0; a < NP; ++a) s_flux[a * G::FALL + G::foff(d) + i] = fl[a];
    }
  }
  __syncthreads();

  // 4. one cell per thread
  if (!inside) return;
  Real ph[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) ph[a] = s_phi[a * G::HC + h];
  if (!multi) {
#pragma unroll
    for (int s = 0; s < NS; ++s) phi_out[s * P.plane + g] = ph[NP == 2 ? 1 : s];
    return;
  }
  Real div[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) div[a] = Real(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int ex = G::fext(d, 0), ey = G::fext(d, 1);
    const int lo = t3[0] + ex * (t3[1] + ey * t3[2]);
    const int up = lo + (d == 0 ? 1 : (d == 1 ? ex : ex * ey));
#pragma unroll
    for (int a = 0; a < NP; ++a)
      div[a] += s_flux[a * G::FALL + G::foff(d) + up] - s_flux[a * G::FALL + G::foff(d) + lo];
  }
  // da/dphi_a = sum_{b != a} gamma_ab dA/dq(q_ab) . grad phi_b (central gradients)
  Real gc[NP][D];
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const int st = G::hstride(t);
      gc[a][t] = Real(0.5) * (s_phi[a * G::HC + h + st] - s_phi[a * G::HC + h - st]);
    }
  Real dadphi[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) dadphi[a] = Real(0);
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int b = a + 1; b < NP; ++b) {
      const Real gab = P.gamma[a][b];
      if (gab == Real(0)) continue;
      Real q[D], v[D];
#pragma unroll
      for (int t = 0; t < D; ++t) q[t] = ph[a] * gc[b][t] - ph[b] * gc[a][t];
      dAdq_vec<D>(q, P.delta[a][b], P.q_floor, v);
      Real va = Real(0), vb = Real(0);
#pragma unroll
      for (int t = 0; t < D; ++t) {
        va += v[t] * gc[b][t];
        vb += v[t] * gc[a][t];
      }
      dadphi[a] += gab * va;
      dadphi[b] -= gab * vb;
    }
  // grand potentials psi_b(mu, T), theta = T - T_E
  Real mu[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) mu[i] = mu_in[i * P.plane + g];
  const int v_coord = D == 3 ? gz : gy;
  const Real theta = (Real(P.theta0) - Real(P.GV) * Real(clock[0])) + P.G * Real(v_coord);
  Real psi[NP];
#pragma unroll
  for (int b = 0; b < NP; ++b) {
    Real s = P.S[b] * theta;
#pragma unroll
    for (int i = 0; i < NC; ++i) s -= mu[i] * mu[i] * P.inv4A[b] + mu[i] * P.ceq[b][i];
    psi[b] = s;
  }
  // unconstrained rates g_a
  Real rate[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    Real obst = Real(0), drive = Real(0);
#pragma unroll
    for (int b = 0; b < NP; ++b) {
      if (b != a) obst += P.gamma[a][b] * ph[b];
      drive += psi[b] * interp_dh<NP>(ph, b, a);
    }
    rate[a] = P.eps * (div[a] - dadphi[a]) - P.obst * obst - drive;
  }
  int na = 0;
  Real lam = Real(0);
#pragma unroll
  for (int a = 0; a < NP; ++a)
    if (act & (1u << a)) {
      lam += rate[a];
      ++na;
    }
  lam = lam / Real(na);
  Real u[NP];
  int m = 0;
#pragma unroll
  for (int a = 0; a < NP; ++a)
    if (act & (1u << a)) u[m++] = ph[a] + P.mob_eps * (rate[a] - lam);
  Real out[NP];
  if (NP == 2) {
    // only phi_1 is stored: clamp it to [0, 1] (the two-phase projection)
    Real s = u[1];
    out[1] = s < Real(0) ? Real(0) : (s > Real(1) ? Real(1) : s);
  } else {
    project_simplex<Real, NP>(u, m);
    m = 0;
#pragma unroll
    for (int a = 0; a < NP; ++a) out[a] = (act & (1u << a)) ? u[m++] : Real(0);
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) phi_out[s * P.plane + g] = out[NP == 2 ? 1 : s];
}

// ------------------------------------------------------------------ mu + LBM
template <int D, int NP, int NC, class Real>
struct MlSmem {
  using G = Geo<D, Real>;
  static constexpr int Q = D == 2 ? 9 : 19;
  static constexpr size_t po = 0;                                   // phi^n
  static constexpr size_t pn = po + sizeof(Real) * NP * G::HC;      // phi^{n+1}
  static constexpr size_t mu = pn + sizeof(Real) * NP * G::HC;      // mu^n
  static constexpr size_t u = mu + sizeof(Real) * NC * G::HC;       // U^n
  static constexpr size_t hl = u + sizeof(Real) * D * G::HC;        // h_liquid(phi^{n+1})
  static constexpr size_t fs = hl + sizeof(Real) * G::HC;           // collided deviations
  static constexpr size_t J = fs + sizeof(Real) * Q * G::HC;        // face fluxes
  static constexpr size_t chg = J + sizeof(Real) * NC * G::FALL;    // phi changed
  static constexpr size_t bytes = chg + G::HC + 16;
};

template <int D, int NP, int NC, class Real, class Store>
__global__ void __launch_bounds__(Geo<D, Real>::NT)
    mu_lbm_kernel(const DevParams<Real> P, const Real* __restrict__ phi_old,
                  const Real* __restrict__ phi_new, const Real* __restrict__ mu_in,
                  const Store* __restrict__ f_in, Real* __restrict__ mu_out,
                  Store* __restrict__ f_out, const double* __restrict__ clock_in,
                  double* __restrict__ clock_out) {
  using G = Geo<D, Real>;
  using L = MlSmem<D, NP, NC, Real>;
  using Lat = typename LatticeOf<D>::type;
  constexpr int Q = D == 2 ? 9 : 19;
  extern __shared__ __align__(16) unsigned char smem[];
  Real* s_po = reinterpret_cast<Real*>(smem + L::po);
  Real* s_pn = reinterpret_cast<Real*>(smem + L::pn);
  Real* s_mu = reinterpret_cast<Real*>(smem + L::mu);
  Real* s_u = reinterpret_cast<Real*>(smem + L::u);
  Real* s_hl = reinterpret_cast<Real*>(smem + L::hl);
  Real* s_fs = reinterpret_cast<Real*>(smem + L::fs);
  Real* s_J = reinterpret_cast<Real*>(smem + L::J);
  unsigned char* s_chg = smem + L::chg;

  const int tid = threadIdx.x;
  const int b0[3] = {(int)blockIdx.x * G::TX, (int)blockIdx.y * G::TY, (int)blockIdx.z * G::TZ};
  const bool inner = tile_inside<D>(P, b0);
  const double t_now = clock_in[0];
  const Real theta_base = Real(P.theta0) - Real(P.GV) * Real(t_now);
  const Real omega = Real(1) - P.inv_tau_f;

  // 1. stage phi^n, phi^{n+1}, mu^n on tile + halo; moments of f^n,
  //    rho, U = (m + F_B/2) / (rho (1 + kappa/2)), F = F_B - rho kappa U,
  //    and the BGK + Guo collision of every staged cell
  for (int h = tid; h < G::HC; h += G::NT) {
    int c[3];
    halo_coords<D>(P, b0, inner, h, c);
    const long long g = cell_index<D>(P, c[0], c[1], c[2]);
    Real po[NP], pn[NP];
    load_phases<NP>(phi_old, g, P.plane, po);
    load_phases<NP>(phi_new, g, P.plane, pn);
    bool changed = false;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      s_po[a * G::HC + h] = po[a];
      s_pn[a * G::HC + h] = pn[a];
      changed = changed || (po[a] != pn[a]);
    }
    s_chg[h] = changed ? 1 : 0;
    s_hl[h] = interp_h<NP>(pn, 0);
    Real mu[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      mu[i] = mu_in[i * P.plane + g];
      s_mu[i * G::HC + h] = mu[i];
    }
    Real dk[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) dk[k] = Codec<Store>::load(f_in[k * P.plane + g]);
    Real drho = Real(0), m[D];
#pragma unroll
    for (int a = 0; a < D; ++a) m[a] = Real(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      drho += dk[k];
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (Lat::c(k, a) != 0) m[a] += Real(Lat::c(k, a)) * dk[k];
    }
    const Real rho = Real(1) + drho;
    const Real phil = obstacle(P, c[0], c[1], c[2]) ? Real(0) : po[0];
    const Real sl = Real(1) - phil;
    const Real kappa = P.kappa0 * sl * sl;
    const Real theta = theta_base + P.G * Real(D == 3 ? c[2] : c[1]);
    Real drive = P.gbeta_T * (theta + P.dT_ref);
#pragma unroll
    for (int i = 0; i < NC; ++i) drive += P.gbeta_c[i] * (P.dcl_ref[i] + mu[i] * P.inv2A[0]);
    const Real FB = rho * phil * drive;
    const Real inv = Real(1) / (rho * (Real(1) + Real(0.5) * kappa));
    Real u[D], F[D];
    Real uu = Real(0), uF = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const Real fb = a == D - 1 ? FB : Real(0);
      u[a] = (m[a] + Real(0.5) * fb) * inv;
      F[a] = fb - rho * kappa * u[a];
      s_u[a * G::HC + h] = u[a];
      uu += u[a] * u[a];
      uF += u[a] * F[a];
    }
    // f*_k - w_k = (1 - 1/tau) d_k + (feq_k - w_k)/tau + G_k with
    // feq_k - w_k = w_k [(drho - 1.5 rho U.U) + rho cu (3 + 4.5 cu)],
    // G_k = w_k [-3 (1 - 1/2tau) U.F + (1 - 1/2tau) cF (3 + 9 cu)]
    const Real A0 = drho - Real(1.5) * rho * uu;
    const Real B0 = Real(-3) * P.force_pre * uF;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      Real cu = Real(0), cF = Real(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (Lat::c(k, a) > 0) {
          cu += u[a];
          cF += F[a];
        } else if (Lat::c(k, a) < 0) {
          cu -= u[a];
          cF -= F[a];
        }
      }
      const Real wk = Real(Lat::w(k));
      const Real deq = wk * (A0 + rho * cu * (Real(3) + Real(4.5) * cu));
      const Real Gk = wk * (B0 + P.force_pre * cF * (Real(3) + Real(9) * cu));
      s_fs[k * G::HC + h] = omega * dk[k] + P.inv_tau_f * deq + Gk;
    }
  }
  __syncthreads();

  // 2. solute flux through every face of the tile: diffusion
  //    -M_f (mu_b - mu_a), antitrapping
  //    -a eps sum_{a>0} [phi_l]_f [c_l - c_a]_f [dphi_a]_f n_a.e_d, advection
  //    [U_d h_l c_l]_f; zero through walls and obstacle cells
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int ex = G::fext(d, 0), ey = G::fext(d, 1);
    for (int i = tid; i < G::fcount(d); i += G::NT) {
      const int f[3] = {i % ex, (i / ex) % ey, i / (ex * ey)};
      const int gd = b0[d] + f[d];
      Real J[NC];
#pragma unroll
      for (int s = 0; s < NC; ++s) J[s] = Real(0);
      bool closed = (P.bc[d] == kWall && (gd == 0 || gd == P.n[d])) || gd > P.n[d];
      if (!closed && (P.wall[0] | P.wall[1] | P.wall[2])) {
        int ga[3] = {b0[0] + f[0], b0[1] + f[1], b0[2] + f[2]};
        int gb[3] = {ga[0], ga[1], ga[2]};
        ga[d] -= 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          ga[a] = (a < D) ? fold_axis(P, ga[a], a) : 0;
          gb[a] = (a < D) ? fold_axis(P, gb[a], a) : 0;
        }
        closed = obstacle(P, ga[0], ga[1], ga[2]) || obstacle(P, gb[0], gb[1], gb[2]);
      }
      if (!closed) {
        const int hb = (f[0] + 1) * G::SX + (f[1] + 1) * G::SY + (f[2] + G::ZOFF) * G::SZ;
        const int ha = hb - G::hstride(d);
        const Real Mf = Real(0.5) * P.M0 * (s_pn[ha] + s_pn[hb]);  // plane 0 = liquid
        const Real ua = s_u[d * G::HC + ha] * s_hl[ha], ub = s_u[d * G::HC + hb] * s_hl[hb];
#pragma unroll
        for (int s = 0; s < NC; ++s) {
          const Real ma = s_mu[s * G::HC + ha], mb = s_mu[s * G::HC + hb];
          J[s] = -Mf * (mb - ma) +
                 Real(0.5) * (ua * (P.ceq[0][s] + ma * P.inv2A[0]) + ub * (P.ceq[0][s] + mb * P.inv2A[0]));
        }
        if (P.at_eps != Real(0) && (s_chg[ha] | s_chg[hb])) {
          Real at[NC];
#pragma unroll
          for (int s = 0; s < NC; ++s) at[s] = Real(0);
#pragma unroll
          for (int a = 1; a < NP; ++a) {
            const Real* sp = s_po + a * G::HC;
            Real g2 = Real(0), gn = Real(0);
#pragma unroll
            for (int t = 0; t < D; ++t) {
              Real gt;
              if (t == d) {
                gt = sp[hb] - sp[ha];
                gn = gt;
              } else {
                const int st = G::hstride(t);
                gt = Real(0.25) * (sp[ha + st] + sp[hb + st] - sp[ha - st] - sp[hb - st]);
              }
              g2 += gt * gt;
            }
            if (g2 <= Real(1e-12)) continue;
            // antitrapping acts where liquid is present: weight by phi_l^n on the face
            const Real nd = Real(0.5) * (s_po[ha] + s_po[hb]) * gn / sqrt(g2);
            const Real dphi = Real(0.5) * ((s_pn[a * G::HC + ha] - sp[ha]) + (s_pn[a * G::HC + hb] - sp[hb]));
            const Real dinv = P.inv2A[0] - P.inv2A[a];
#pragma unroll
            for (int s = 0; s < NC; ++s) {
              const Real dc0 = P.ceq[0][s] - P.ceq[a][s];
              const Real dc = dc0 + Real(0.5) * (s_mu[s * G::HC + ha] + s_mu[s * G::HC + hb]) * dinv;
              at[s] += dc * dphi * nd;
            }
          }
#pragma unroll
          for (int s = 0; s < NC; ++s) J[s] -= P.at_eps * at[s];
        }
      }
#pragma unroll
      for (int s = 0; s < NC; ++s) s_J[s * G::FALL + G::foff(d) + i] = J[s];
    }
  }
  __syncthreads();

  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0) clock_out[0] = t_now + 1.0;

  // 3. one cell per thread: mu^{n+1}, then f^{n+1} pulled from the collided
  //    populations of the neighbours (halfway bounce-back on walls)
  const int t3[3] = {tid % G::TX, (tid / G::TX) % G::TY, tid / (G::TX * G::TY)};
  const int gc3[3] = {b0[0] + t3[0], b0[1] + t3[1], b0[2] + t3[2]};
  if (gc3[0] >= P.n[0] || gc3[1] >= P.n[1] || gc3[2] >= P.n[2]) return;
  const long long g = cell_index<D>(P, gc3[0], gc3[1], gc3[2]);
  const int h = (t3[0] + 1) * G::SX + (t3[1] + 1) * G::SY + (t3[2] + G::ZOFF) * G::SZ;

  if (obstacle(P, gc3[0], gc3[1], gc3[2])) {
#pragma unroll
    for (int s = 0; s < NC; ++s) mu_out[s * P.plane + g] = s_mu[s * G::HC + h];
  } else {
    Real po[NP], pn[NP], ho[NP], hn[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      po[a] = s_po[a * G::HC + h];
      pn[a] = s_pn[a * G::HC + h];
    }
    Real chi = Real(0);
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      ho[a] = interp_h<NP>(po, a);
      hn[a] = interp_h<NP>(pn, a);
      chi += hn[a] * P.inv2A[a];
    }
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      const Real mu = s_mu[s * G::HC + h];
      Real div = Real(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int ex = G::fext(d, 0), ey = G::fext(d, 1);
        const int lo = t3[0] + ex * (t3[1] + ey * t3[2]);
        const int up = lo + (d == 0 ? 1 : (d == 1 ? ex : ex * ey));
        div += s_J[s * G::FALL + G::foff(d) + up] - s_J[s * G::FALL + G::foff(d) + lo];
      }
      Real src = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) src += (P.ceq[a][s] + mu * P.inv2A[a]) * (hn[a] - ho[a]);
      mu_out[s * P.plane + g] = mu + (-div - src) / chi;
    }
  }

#pragma unroll
  for (int k = 0; k < Q; ++k) {
    bool bounce = false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int sa = gc3[a] - Lat::c(k, a);
      if (P.bc[a] == kWall && (sa < 0 || sa >= P.n[a])) bounce = true;
    }
    const int hs = h - Lat::c(k, 0) * G::SX - Lat::c(k, 1) * G::SY - (D == 3 ? Lat::c(k, 2) * G::SZ : 0);
    const Real v = bounce ? s_fs[Lat::opp(k) * G::HC + h] : s_fs[k * G::HC + hs];
    f_out[k * P.plane + g] = Codec<Store>::put(v);
  }
}

// ------------------------------------------------------------------ state I/O
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

// Exchange-format fields of the current state; any output may be null.
// phi: N planes (liquid first); c_i = sum_a h_a (ceq_a,i + mu_i / (2 A_a));
// f = w + d; rho = 1 + sum d; U as in the step (force-corrected); dev = d.
template <int D, int NP, int NC, class Real, class Store, class Out>
__global__ void fields_kernel(const DevParams<Real> P, const Real* __restrict__ phi,
                              const Real* __restrict__ mu_in, const Store* __restrict__ f,
                              const double* __restrict__ clock, Out* __restrict__ o_phi,
                              Out* __restrict__ o_mu, Out* __restrict__ o_c, Out* __restrict__ o_f,
                              Out* __restrict__ o_rho, Out* __restrict__ o_u,
                              Out* __restrict__ o_dev) {
  using Lat = typename LatticeOf<D>::type;
  constexpr int Q = D == 2 ? 9 : 19;
  const long long cells = (long long)P.n[0] * P.n[1] * P.n[2];
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (x >= cells) return;
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
  if (o_c) {
    Real h[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) h[a] = interp_h<NP>(p, a);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      Real c = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) c += h[a] * (P.ceq[a][i] + mu[i] * P.inv2A[a]);
      o_c[i * cells + x] = Out(c);
    }
  }
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
    const int v_coord = D == 3 ? gz : gy;
    const Real theta = Real(P.theta0 - P.GV * clock[0]) + P.G * Real(v_coord);
    Real drive = P.gbeta_T * (theta + P.dT_ref);
#pragma unroll
    for (int i = 0; i < NC; ++i) drive += P.gbeta_c[i] * (P.dcl_ref[i] + mu[i] * P.inv2A[0]);
    const Real FB = rho * phil * drive;
    const Real inv = Real(1) / (rho * (Real(1) + Real(0.5) * kappa));
#pragma unroll
    for (int a = 0; a < D; ++a) o_u[a * cells + x] = Out((m[a] + (a == D - 1 ? Real(0.5) * FB : Real(0))) * inv);
  }
}

// ------------------------------------------------------------------ invariants
// Per-cell totals in FP64 without fused multiply-add, in a fixed order, and
// a fixed-order block reduction (see gpflbm_invariants in gpflbm.h).
struct InvParams {
  long long cells, plane;
  int nx, px;
  double ceq[4][2];
  double inv2A[4];
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
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      double c = 0.0;
#pragma unroll
      for (int a = 0; a < NP; ++a)
        c = __dadd_rn(c, __dmul_rn(h[a], __dadd_rn(P.ceq[a][i], __dmul_rn(m[i], P.inv2A[a]))));
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

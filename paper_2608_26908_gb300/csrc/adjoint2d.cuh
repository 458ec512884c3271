// Hand-written discrete adjoint of the 2D step for two phases and one solute
// (D2Q9), the configuration of the differentiation workload.
//
// With phi_l = 1 - s (s = phi_1) the phase-field update of a cell whose 3x3
// neighbourhood holds both phases is
//   u = s + (mob/2) [ gamma D(s) - c_ob (1 - 2 s) - (6/eps) s (1-s) dpsi ],
//   s' = clamp(u, 0, 1),
// D = sum_d V_d(x+e_d/2) - V_d(x-e_d/2), V_d(face) = dA/dq_d at q = grad_f s,
// c_ob = 16 gamma / (pi^2 eps^2), dpsi = psi_1 - psi_0 (the centre terms
// da/dphi cancel between the two phases).  Elsewhere s' = s.  The adjoint
// takes the derivative of exactly this piecewise map: zero through a clamped
// cell (the active-set subgradient), the identity for single-phase cells.
//
// One backward step n+1 -> n (S^n, S^{n+1} recomputed and stored):
//   adj_mu_face_kernel  per cell: the adjoint coefficients of its +x and +y
//                       solute faces (diffusion, advection, antitrapping);
//                       antitrapping's transverse terms go out by atomics;
//   adj_cell_kernel     per cell: gathers its faces, the mu-stage terms
//                       (chi', source), the BGK + Guo collision and moment
//                       (drag, buoyancy) adjoint of its populations pulled
//                       back along c_k, and the clamp; writes lambda_mu^n,
//                       lambda_f^n, part of lambda_s^n and lambda_u;
//   adj_pf_face_kernel  per cell: the phase-field faces (Hessian of A by dual
//                       numbers) scattered to the six cells they read.
// Parameter gradients (mobility, delta, g beta_c) accumulate per cell in FP64.
#pragma once

#include "gpflbm_kernels.cuh"

namespace gpflbm {

// value + tangent, for exact derivatives of the gradient-energy flux
template <class Real>
struct Tan {
  Real v, d;
  __device__ Tan(Real a = Real(0), Real b = Real(0)) : v(a), d(b) {}
};
template <class Real>
__device__ __forceinline__ Tan<Real> operator+(Tan<Real> a, Tan<Real> b) {
  return Tan<Real>(a.v + b.v, a.d + b.d);
}
template <class Real>
__device__ __forceinline__ Tan<Real> operator-(Tan<Real> a, Tan<Real> b) {
  return Tan<Real>(a.v - b.v, a.d - b.d);
}
template <class Real>
__device__ __forceinline__ Tan<Real> operator*(Tan<Real> a, Tan<Real> b) {
  return Tan<Real>(a.v * b.v, a.d * b.v + a.v * b.d);
}
template <class Real>
__device__ __forceinline__ Tan<Real> operator/(Tan<Real> a, Tan<Real> b) {
  return Tan<Real>(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}

// dA/dq_j of the cubic-anisotropy gradient energy in tangent arithmetic
// (same formula and floor rule as the forward dAdq)
template <class Real>
__device__ __forceinline__ Tan<Real> dAdq_tan(const Tan<Real>* q, Tan<Real> delta, Real q_floor, int j) {
  const Tan<Real> s2 = q[0] * q[0] + q[1] * q[1];
  const Tan<Real> s4 = q[0] * q[0] * q[0] * q[0] + q[1] * q[1] * q[1] * q[1];
  if (s2.v <= q_floor) return Tan<Real>(Real(2)) * q[j];
  const Tan<Real> inv2 = Tan<Real>(Real(1)) / s2;
  const Tan<Real> r4 = s4 * inv2 * inv2;
  const Tan<Real> ac = Tan<Real>(Real(1)) - delta * (Tan<Real>(Real(3)) - Tan<Real>(Real(4)) * r4);
  const Tan<Real> qj = q[j];
  const Tan<Real> dac = Tan<Real>(Real(16)) * delta * (qj * qj * qj - qj * s4 * inv2) * inv2 * inv2;
  return Tan<Real>(Real(2)) * ac * (ac * qj + s2 * dac);
}

// H(s) = s^2 (3 - 2 s) and H'(s) = 6 s (1 - s): h_1 for two phases
template <class Real>
__device__ __forceinline__ Real Hs(Real s) { return s * s * (Real(3) - Real(2) * s); }
template <class Real>
__device__ __forceinline__ Real dHs(Real s) { return Real(6) * s * (Real(1) - s); }

template <class Real>
struct AdjIO {
  const Real* s0;    // S^n: phi_1 (internal layout)
  const Real* mu0;   //      mu
  const Real* d0;    //      f - w (9 planes)
  const Real* s1;    // S^{n+1}: phi_1
  const Real* mu1;   //          mu
  const Real* ls1;   // adjoint of S^{n+1}
  const Real* lmu1;
  const Real* ld1;
  Real* ls0;         // adjoint of S^n (ls0 accumulates; zeroed before the step)
  Real* lmu0;
  Real* ld0;
  Real* mface;       // solute-face coefficients: 2 faces x 8 values per cell
  Real* lu;          // lambda of the unclamped phase-field value u
  double* gacc;      // parameter-gradient accumulators: 3 planes (mob, delta, gbeta)
  const double* clock;  // time of step n (device)
};

constexpr int kMF = 8;  // per solute face: cmu_a, cmu_b, csp_a, csp_b, cU_a, cU_b, cs_a, cs_b

// rho, U and F of a cell from S^n (the forward moment computation)
template <class Real>
struct Macro2 {
  Real drho, rho, mx, my, phil, kappa, B, FB, iv, ux, uy, Fx, Fy;
};

template <class Real>
__device__ __forceinline__ Macro2<Real> macro2(const DevParams<Real>& P, const Real* d, Real s, Real mu,
                                               bool obs, Real theta) {
  Macro2<Real> m;
  m.drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
  m.mx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
  m.my = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
  m.rho = Real(1) + m.drho;
  m.phil = obs ? Real(0) : Real(1) - s;
  const Real sl = Real(1) - m.phil;
  m.kappa = P.kappa0 * sl * sl;
  m.B = P.gbeta_T * (theta + P.dT_ref) + P.gbeta_c[0] * (P.dcl_ref[0] + mu * P.inv2A[0]);
  m.FB = m.rho * m.phil * m.B;
  m.iv = Real(1) / (m.rho * (Real(1) + Real(0.5) * m.kappa));
  m.ux = m.mx * m.iv;
  m.uy = (m.my + Real(0.5) * m.FB) * m.iv;
  m.Fx = -m.rho * m.kappa * m.ux;
  m.Fy = m.FB - m.rho * m.kappa * m.uy;
  return m;
}

template <class Real>
__device__ __forceinline__ void cell_xy(const DevParams<Real>& P, long long c, int* x, int* y) {
  *x = (int)(c % P.n[0]);
  *y = (int)(c / P.n[0]);
}

template <class Real>
__device__ __forceinline__ long long off2(const DevParams<Real>& P, int x, int y) {
  return (long long)y * P.px + x;
}

// A(x) = lambda_mu^{n+1} / chi'(x) (0 in obstacle cells)
template <class Real>
__device__ __forceinline__ Real adj_A(const DevParams<Real>& P, const AdjIO<Real>& io, long long o, bool obs) {
  if (obs) return Real(0);
  const Real e = P.inv2A[1] - P.inv2A[0];
  const Real chi = P.inv2A[0] + Hs(io.s1[o]) * e;
  return io.lmu1[o] / chi;
}

template <class Real>
__global__ void __launch_bounds__(256) adj_mu_face_kernel(const DevParams<Real> P, const AdjIO<Real> io) {
  const long long cells = (long long)P.n[0] * P.n[1];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= cells) return;
  int x, y;
  cell_xy(P, c, &x, &y);
  const long long oa = off2(P, x, y);
  const bool walls = (P.wall[0] | P.wall[1]) != 0;
  const bool obsA = walls && obstacle(P, x, y, 0);
  const Real theta_base = Real(P.theta0) - Real(P.GV) * Real(io.clock[0]);
  const Real A_a = adj_A(P, io, oa, obsA);
  Real da[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) da[k] = io.d0[k * P.plane + oa];
  const Macro2<Real> ma = macro2(P, da, io.s0[oa], io.mu0[oa], obsA, theta_base + P.G * Real(y));
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    Real cf[kMF];
#pragma unroll
    for (int j = 0; j < kMF; ++j) cf[j] = Real(0);
    const int bxr = d == 0 ? x + 1 : x, byr = d == 0 ? y : y + 1;
    const int gbd = d == 0 ? bxr : byr;
    bool closed = P.bc[d] == kWall && gbd == P.n[d];
    const int bx = fold_axis(P, bxr, 0), by = fold_axis(P, byr, 1);
    const bool obsB = walls && obstacle(P, bx, by, 0);
    closed = closed || obsA || obsB;
    if (!closed) {
      const long long ob = off2(P, bx, by);
      const Real A_b = adj_A(P, io, ob, obsB);
      const Real L = A_b - A_a;  // adjoint of the face flux
      Real db[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) db[k] = io.d0[k * P.plane + ob];
      const Macro2<Real> mb = macro2(P, db, io.s0[ob], io.mu0[ob], obsB, theta_base + P.G * Real(by));
      const Real s0a = io.s0[oa], s0b = io.s0[ob], s1a = io.s1[oa], s1b = io.s1[ob];
      const Real mua = io.mu0[oa], mub = io.mu0[ob];
      const Real Mf = Real(0.5) * P.M0 * ((Real(1) - s1a) + (Real(1) - s1b));
      // diffusion -M_f (mu_b - mu_a), M = M0 (1 - s')
      cf[0] += L * Mf;
      cf[1] -= L * Mf;
      cf[2] += L * Real(0.5) * P.M0 * (mub - mua);
      cf[3] += L * Real(0.5) * P.M0 * (mub - mua);
      // advection 1/2 [U_d h0' c0(mu)]_a + [...]_b, h0' = 1 - H(s')
      const Real ua = d == 0 ? ma.ux : ma.uy, ub = d == 0 ? mb.ux : mb.uy;
      const Real h0a = Real(1) - Hs(s1a), h0b = Real(1) - Hs(s1b);
      const Real c0a = P.ceq[0][0] + mua * P.inv2A[0], c0b = P.ceq[0][0] + mub * P.inv2A[0];
      cf[4] += L * Real(0.5) * h0a * c0a;
      cf[5] += L * Real(0.5) * h0b * c0b;
      cf[0] += L * Real(0.5) * ua * h0a * P.inv2A[0];
      cf[1] += L * Real(0.5) * ub * h0b * P.inv2A[0];
      cf[2] -= L * Real(0.5) * ua * c0a * dHs(s1a);
      cf[3] -= L * Real(0.5) * ub * c0b * dHs(s1b);
      // antitrapping -a eps liq dc dphi nd
      if (P.at_eps != Real(0)) {
        const int st_x = d == 0 ? 0 : 1, st_y = d == 0 ? 1 : 0;  // transverse unit step
        const int ap_x = fold_axis(P, x + st_x, 0), ap_y = fold_axis(P, y + st_y, 1);
        const int am_x = fold_axis(P, x - st_x, 0), am_y = fold_axis(P, y - st_y, 1);
        const int bp_x = fold_axis(P, bxr + st_x, 0), bp_y = fold_axis(P, byr + st_y, 1);
        const int bm_x = fold_axis(P, bxr - st_x, 0), bm_y = fold_axis(P, byr - st_y, 1);
        const long long oap = off2(P, ap_x, ap_y), oam = off2(P, am_x, am_y);
        const long long obp = off2(P, bp_x, bp_y), obm = off2(P, bm_x, bm_y);
        const Real gn = s0b - s0a;
        const Real gt = Real(0.25) * (io.s0[oap] + io.s0[obp] - io.s0[oam] - io.s0[obm]);
        const Real g2 = gn * gn + gt * gt;
        if (g2 > Real(1e-12)) {
          const Real rg = Real(1) / sqrt(g2);
          const Real nd = gn * rg;
          const Real liq = Real(1) - Real(0.5) * (s0a + s0b);
          const Real dinv = P.inv2A[0] - P.inv2A[1];
          const Real dc = (P.ceq[0][0] - P.ceq[1][0]) + Real(0.5) * (mua + mub) * dinv;
          const Real dphi = Real(0.5) * ((s1a - s0a) + (s1b - s0b));
          const Real k = -P.at_eps * L;
          const Real jl = k * dc * dphi * nd;   // d/d liq
          const Real jc = k * liq * dphi * nd;  // d/d dc
          const Real jp = k * liq * dc * nd;    // d/d dphi
          const Real jn = k * liq * dc * dphi;  // d/d nd
          const Real dn_gn = gt * gt * rg * rg * rg;
          const Real dn_gt = -gn * gt * rg * rg * rg;
          cf[6] += -Real(0.5) * jl - Real(0.5) * jp - jn * dn_gn;
          cf[7] += -Real(0.5) * jl - Real(0.5) * jp + jn * dn_gn;
          cf[2] += Real(0.5) * jp;
          cf[3] += Real(0.5) * jp;
          cf[0] += Real(0.5) * dinv * jc;
          cf[1] += Real(0.5) * dinv * jc;
          const Real T = Real(0.25) * jn * dn_gt;
          atomicAdd(io.ls0 + oap, T);
          atomicAdd(io.ls0 + obp, T);
          atomicAdd(io.ls0 + oam, -T);
          atomicAdd(io.ls0 + obm, -T);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMF; ++j) io.mface[(d * kMF + j) * P.plane + oa] = cf[j];
  }
}

template <class Real>
__global__ void __launch_bounds__(256) adj_cell_kernel(const DevParams<Real> P, const AdjIO<Real> io) {
  using Lat = Lattice<9>;
  const long long cells = (long long)P.n[0] * P.n[1];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= cells) return;
  int x, y;
  cell_xy(P, c, &x, &y);
  const int nx = P.n[0], ny = P.n[1];
  const long long o = off2(P, x, y);
  const bool walls = (P.wall[0] | P.wall[1]) != 0;
  const bool obs = walls && obstacle(P, x, y, 0);
  const Real theta = Real(P.theta0) - Real(P.GV) * Real(io.clock[0]) + P.G * Real(y);
  const Real s0 = io.s0[o], s1 = io.s1[o], mu0 = io.mu0[o], mu1 = io.mu1[o];
  const Real e = P.inv2A[1] - P.inv2A[0];

  Real lmu = Real(0), ls = Real(0), lsp = io.ls1[o], gUx = Real(0), gUy = Real(0);
  // solute faces: this cell is a of its +x/+y faces and b of the faces below
  if (!obs) {
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const Real* fa = io.mface + (d * kMF) * P.plane;
      lmu += fa[0 * P.plane + o];
      lsp += fa[2 * P.plane + o];
      ls += fa[6 * P.plane + o];
      const Real ua = fa[4 * P.plane + o];
      if (d == 0) gUx += ua; else gUy += ua;
      const int lx = d == 0 ? x - 1 : x, ly = d == 0 ? y : y - 1;
      const bool has_lower = P.bc[d] != kWall || (d == 0 ? x > 0 : y > 0);
      if (has_lower) {
        const long long ol = off2(P, fold_axis(P, lx, 0), fold_axis(P, ly, 1));
        lmu += fa[1 * P.plane + ol];
        lsp += fa[3 * P.plane + ol];
        ls += fa[7 * P.plane + ol];
        const Real ub = fa[5 * P.plane + ol];
        if (d == 0) gUx += ub; else gUy += ub;
      }
    }
  }
  // mu update: mu' = mu + (-div J - src) / chi', src = (c1 - c0)(mu) (H(s') - H(s))
  if (obs) {
    lmu += io.lmu1[o];
  } else {
    const Real chi = P.inv2A[0] + Hs(s1) * e;
    const Real A = io.lmu1[o] / chi;
    const Real dH = Hs(s1) - Hs(s0);
    lmu += io.lmu1[o] - A * e * dH;
    const Real c10 = (P.ceq[1][0] - P.ceq[0][0]) + mu0 * e;
    lsp += -A * c10 * dHs(s1) + (-A * (mu1 - mu0)) * e * dHs(s1);
    ls += A * c10 * dHs(s0);
  }
  // populations: pull transposed (bounce-back at walls), then BGK + Guo
  Real dk[9], a[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    dk[k] = io.d0[k * P.plane + o];
    const int cx = Lat::c(k, 0), cy = Lat::c(k, 1);
    int tx = x + cx, ty = y + cy;
    const bool bounce = (P.bc[0] == kWall && (tx < 0 || tx >= nx)) || (P.bc[1] == kWall && (ty < 0 || ty >= ny));
    if (bounce) {
      a[k] = io.ld1[Lat::opp(k) * P.plane + o];
    } else {
      tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
      ty = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
      a[k] = io.ld1[k * P.plane + off2(P, tx, ty)];
    }
  }
  const Macro2<Real> m = macro2(P, dk, s0, mu0, obs, theta);
  const Real omega = Real(1) - P.inv_tau_f, pre = P.force_pre, itau = P.inv_tau_f;
  const Real uu = m.ux * m.ux + m.uy * m.uy;
  Real gr = Real(0), gFx = Real(0), gFy = Real(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const Real cx = Real(Lat::c(k, 0)), cy = Real(Lat::c(k, 1)), wk = Real(Lat::w(k));
    const Real cu = cx * m.ux + cy * m.uy, cF = cx * m.Fx + cy * m.Fy;
    const Real ak = a[k];
    // deq/tau: (w/tau)(drho - 1.5 rho U.U + rho cu (3 + 4.5 cu))
    gr += ak * wk * itau * (Real(1) - Real(1.5) * uu + cu * (Real(3) + Real(4.5) * cu));
    const Real gcu = ak * wk * (itau * m.rho * (Real(3) + Real(9) * cu) + pre * Real(9) * cF);
    gUx += ak * wk * itau * (-Real(3) * m.rho * m.ux) + gcu * cx + ak * wk * (-Real(3) * pre * m.Fx);
    gUy += ak * wk * itau * (-Real(3) * m.rho * m.uy) + gcu * cy + ak * wk * (-Real(3) * pre * m.Fy);
    const Real gcF = ak * wk * pre * (Real(3) + Real(9) * cu);
    gFx += ak * wk * (-Real(3) * pre * m.ux) + gcF * cx;
    gFy += ak * wk * (-Real(3) * pre * m.uy) + gcF * cy;
  }
  // F = F_B e_y - rho kappa U;  U = (m + F_B/2 e_y) iv;  iv = 1/(rho (1 + kappa/2))
  gUx += -m.rho * m.kappa * gFx;
  gUy += -m.rho * m.kappa * gFy;
  gr += -m.kappa * (m.ux * gFx + m.uy * gFy);
  Real gk = -m.rho * (m.ux * gFx + m.uy * gFy);
  Real gFB = gFy;
  const Real gmx = gUx * m.iv, gmy = gUy * m.iv;
  gFB += Real(0.5) * gUy * m.iv;
  const Real giv = gUx * m.mx + gUy * (m.my + Real(0.5) * m.FB);
  gr += giv * (-m.iv / m.rho);
  gk += giv * (-Real(0.5) * m.rho * m.iv * m.iv);
  // F_B = rho phil B
  gr += gFB * m.phil * m.B;
  const Real gphil = gFB * m.rho * m.B + gk * (-Real(2) * P.kappa0 * (Real(1) - m.phil));
  const Real gB = gFB * m.rho * m.phil;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const Real cx = Real(Lat::c(k, 0)), cy = Real(Lat::c(k, 1));
    io.ld0[k * P.plane + o] = omega * a[k] + gr + cx * gmx + cy * gmy;
  }
  if (!obs) ls += -gphil;  // phil = 1 - s
  lmu += gB * P.gbeta_c[0] * P.inv2A[0];
  io.gacc[2 * P.plane + o] += (double)(gB * (P.dcl_ref[0] + mu0 * P.inv2A[0]));

  // phase field: s' = clamp(u) where both phases are present, s' = s elsewhere
  bool multi = false;
  if (!obs) {
    unsigned act = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const Real v = io.s0[off2(P, fold_axis(P, x + dx, 0), fold_axis(P, y + dy, 1))];
        if (v > Real(0)) act |= 2u;
        if (Real(1) - v > Real(0)) act |= 1u;
      }
    multi = act == 3u;
  }
  Real lu = Real(0);
  if (multi) {
    if (s1 > Real(0) && s1 < Real(1)) {
      lu = lsp;
      const Real mob = P.mob_eps * P.eps;  // 1 / tau_phi
      const Real dpsi = -mu0 * mu0 * (P.inv4A[1] - P.inv4A[0]) - mu0 * (P.ceq[1][0] - P.ceq[0][0]) +
                        (P.S[1] - P.S[0]) * theta;
      const Real dpsi_dmu = -mu0 * e - (P.ceq[1][0] - P.ceq[0][0]);
      const Real cob = P.obst * P.gamma[0][1] / P.eps;  // 16 gamma / (pi^2 eps^2)
      ls += lu * (Real(1) + Real(0.5) * mob *
                                (Real(2) * cob - (Real(6) / P.eps) * (Real(1) - Real(2) * s0) * dpsi));
      lmu += lu * Real(0.5) * mob * (-(Real(6) / P.eps) * s0 * (Real(1) - s0) * dpsi_dmu);
      io.gacc[0 * P.plane + o] += (double)(lu * (s1 - s0) / mob);
    }
  } else {
    ls += lsp;
  }
  io.lu[o] = lu;
  io.lmu0[o] = lmu;
  io.ls0[o] += ls;
}

// Phase-field faces: lambda_V = (mob/2) gamma (lu(a) - lu(b)) through
// V_d = dA/dq_d(grad_f s) to the six cells of the face stencil.
template <class Real>
__global__ void __launch_bounds__(256) adj_pf_face_kernel(const DevParams<Real> P, const AdjIO<Real> io) {
  const long long cells = (long long)P.n[0] * P.n[1];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= cells) return;
  int x, y;
  cell_xy(P, c, &x, &y);
  const long long oa = off2(P, x, y);
  const Real mob = P.mob_eps * P.eps;
  const Real gam = P.gamma[0][1];
  const Real lua = io.lu[oa];
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const int bxr = d == 0 ? x + 1 : x, byr = d == 0 ? y : y + 1;
    const int gbd = d == 0 ? bxr : byr;
    if (P.bc[d] == kWall && gbd == P.n[d]) continue;  // closed face
    const long long ob = off2(P, fold_axis(P, bxr, 0), fold_axis(P, byr, 1));
    const Real lV = Real(0.5) * mob * gam * (lua - io.lu[ob]);
    if (lV == Real(0)) continue;
    const int st_x = d == 0 ? 0 : 1, st_y = d == 0 ? 1 : 0;
    const long long oap = off2(P, fold_axis(P, x + st_x, 0), fold_axis(P, y + st_y, 1));
    const long long oam = off2(P, fold_axis(P, x - st_x, 0), fold_axis(P, y - st_y, 1));
    const long long obp = off2(P, fold_axis(P, bxr + st_x, 0), fold_axis(P, byr + st_y, 1));
    const long long obm = off2(P, fold_axis(P, bxr - st_x, 0), fold_axis(P, byr - st_y, 1));
    const Real gn = io.s0[ob] - io.s0[oa];
    const Real gt = Real(0.25) * (io.s0[oap] + io.s0[obp] - io.s0[oam] - io.s0[obm]);
    // q[d] = gn, q[1-d] = gt; tangents of V_d along q_d, q_{1-d} and delta
    Real dV[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Tan<Real> q[2];
      q[d] = Tan<Real>(gn, j == 0 ? Real(1) : Real(0));
      q[1 - d] = Tan<Real>(gt, j == 1 ? Real(1) : Real(0));
      const Tan<Real> dl(P.delta[0][1], j == 2 ? Real(1) : Real(0));
      dV[j] = dAdq_tan<Real>(q, dl, P.q_floor, d).d;
    }
    const Real cn = lV * dV[0], ct = Real(0.25) * lV * dV[1];
    atomicAdd(io.ls0 + ob, cn);
    atomicAdd(io.ls0 + oa, -cn);
    atomicAdd(io.ls0 + oap, ct);
    atomicAdd(io.ls0 + obp, ct);
    atomicAdd(io.ls0 + oam, -ct);
    atomicAdd(io.ls0 + obm, -ct);
    io.gacc[1 * P.plane + oa] += (double)(lV * dV[2]);
  }
}

// lambda of the final state from J = w_frac mean_x H(s) + w_tip tip / nx:
// lambda_s = w_frac H'(s) / cells, lambda_mu = lambda_f = 0; gacc cleared.
template <class Real>
__global__ void adj_init_kernel(const DevParams<Real> P, const Real* __restrict__ s, Real wfrac,
                                Real* __restrict__ ls, Real* __restrict__ lmu, Real* __restrict__ ld,
                                double* __restrict__ gacc) {
  const long long cells = (long long)P.n[0] * P.n[1];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= cells) return;
  int x, y;
  cell_xy(P, c, &x, &y);
  const long long o = off2(P, x, y);
  ls[o] = wfrac * dHs(s[o]) / Real(cells);
  lmu[o] = Real(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) ld[k * P.plane + o] = Real(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) gacc[j * P.plane + o] = 0.0;
}

// Soft-argmax tip along the +x ray from (x0, y0): tip = sum_r r p_r with
// p = softmax(kappa r s(r)); adds w_tip/nx d tip / d s to lambda_s and
// writes tip (one block).
template <class Real>
__global__ void adj_tip_kernel(const DevParams<Real> P, const Real* __restrict__ s, int x0, int y0,
                               double kappa, double wtip, Real* __restrict__ ls, double* __restrict__ tip_out) {
  __shared__ double red[256];
  const int nr = P.n[0] - x0;
  const int tid = threadIdx.x;
  double mx = -1e300;
  for (int r = tid; r < nr; r += blockDim.x) mx = fmax(mx, kappa * r * (double)s[off2(P, x0 + r, y0)]);
  red[tid] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
    __syncthreads();
  }
  mx = red[0];
  __syncthreads();
  double num = 0.0, den = 0.0;
  for (int r = tid; r < nr; r += blockDim.x) {
    const double ez = exp(kappa * r * (double)s[off2(P, x0 + r, y0)] - mx);
    num += r * ez;
    den += ez;
  }
  red[tid] = num;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  num = red[0];
  __syncthreads();
  red[tid] = den;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  den = red[0];
  const double tip = num / den;
  if (tid == 0) *tip_out = tip;
  for (int r = tid; r < nr; r += blockDim.x) {
    const long long o = off2(P, x0 + r, y0);
    const double p = exp(kappa * r * (double)s[o] - mx) / den;
    ls[o] += (Real)(wtip / P.n[0] * p * (r - tip) * kappa * r);
  }
}

// Fixed-order sum of a double plane over the cells: per-block partials.
template <class Real>
__global__ void __launch_bounds__(kRedThreads) adj_sum_kernel(const DevParams<Real> P, const double* __restrict__ v,
                                                              double* __restrict__ partial) {
  const long long cells = (long long)P.n[0] * P.n[1];
  double acc = 0.0;
  for (long long c = blockIdx.x * (long long)kRedThreads + threadIdx.x; c < cells;
       c += (long long)gridDim.x * kRedThreads) {
    int x, y;
    cell_xy(P, c, &x, &y);
    acc += v[off2(P, x, y)];
  }
  __shared__ double s_w[kRedThreads / 32];
  const double w = warp_sum_butterfly(acc);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = s_w[0];
    for (int i = 1; i < kRedThreads / 32; ++i) s += s_w[i];
    partial[blockIdx.x] = s;
  }
}

// Fixed-order partial sums of H(s) = h_1 over the cells (solid fraction).
template <class Real>
__global__ void __launch_bounds__(kRedThreads) adj_frac_kernel(const DevParams<Real> P, const Real* __restrict__ s,
                                                               double* __restrict__ partial) {
  const long long cells = (long long)P.n[0] * P.n[1];
  double acc = 0.0;
  for (long long c = blockIdx.x * (long long)kRedThreads + threadIdx.x; c < cells;
       c += (long long)gridDim.x * kRedThreads) {
    int x, y;
    cell_xy(P, c, &x, &y);
    acc += (double)Hs(s[off2(P, x, y)]);
  }
  __shared__ double s_w[kRedThreads / 32];
  const double w = warp_sum_butterfly(acc);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = s_w[0];
    for (int i = 1; i < kRedThreads / 32; ++i) t += s_w[i];
    partial[blockIdx.x] = t;
  }
}

// lambda_mu^0 to the exchange layout (x fastest, no padding)
template <class Real>
__global__ void adj_export_kernel(const DevParams<Real> P, const Real* __restrict__ src, Real* __restrict__ dst) {
  const long long cells = (long long)P.n[0] * P.n[1];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= cells) return;
  int x, y;
  cell_xy(P, c, &x, &y);
  dst[c] = src[off2(P, x, y)];
}

}  // namespace gpflbm

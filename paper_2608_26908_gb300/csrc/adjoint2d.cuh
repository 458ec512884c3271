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
// One backward step n+1 -> n is one launch of adj2d_kernel.  A CTA owns an
// OX x OY tile of output cells and stages, for the tile plus a two-cell
// halo, the per-cell values the faces read (s^n, s^{n+1}, mu^n,
// A = lambda_mu^{n+1} / chi(s^{n+1}), the velocity U^n).  Then, in shared
// memory:
//   1. the adjoint coefficients of every solute face touching the tile plus
//      a one-cell halo (diffusion, advection, antitrapping);
//   2. per cell of the tile plus halo, lambda of the unclamped phase value
//      (lu); per output cell, the faces gathered, the mu-stage terms (chi',
//      source), and the BGK + Guo collision and moment (drag, buoyancy)
//      adjoint of its populations pulled back along c_k;
//   3. the phase-field faces (Hessian of A by tangent arithmetic), gathered
//      by the output cells.
// Every contribution is gathered by the cell that receives it, in a fixed
// order, so the result is the same from run to run.  Where a wall mirrors
// the transverse stencil of a face, the cell next to the wall collects the
// mirrored terms explicitly.  Parameter gradients (mobility, delta,
// g beta_c) accumulate per cell in FP64.
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

// dA/dq_j with the crystal axes turned by theta about z (c = cos, s = sin):
// A of the crystal-frame components r = (c q_x + s q_y, -s q_x + c q_y),
// dA/dq = (c r'_x - s r'_y, s r'_x + c r'_y), r' = dA/dr (as the forward)
template <class Real>
__device__ __forceinline__ Tan<Real> dAdq_tan_tilted(const Tan<Real>* q, Tan<Real> delta, Real c, Real s,
                                                     Real q_floor, int j) {
  const Tan<Real> C(c), S(s);
  Tan<Real> r[2];
  r[0] = C * q[0] + S * q[1];
  r[1] = C * q[1] - S * q[0];
  const Tan<Real> a0 = dAdq_tan<Real>(r, delta, q_floor, 0), a1 = dAdq_tan<Real>(r, delta, q_floor, 1);
  return j == 0 ? C * a0 - S * a1 : S * a0 + C * a1;
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
  Real* ls0;         // adjoint of S^n (written)
  Real* lmu0;
  Real* ld0;
  double* gacc;      // parameter-gradient accumulators: 3 planes (mob, delta, gbeta)
  const double* clock;  // time of step n (device)
};

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
  // c_l - c_ref with ceq_l(T) = ceq_l + dceq_dT (T - T_E)
  m.B = P.gbeta_T * (theta + P.dT_ref) +
        P.gbeta_c[0] * (P.dcl_ref[0] + P.dceq_dT[0][0] * theta + mu * P.inv2A[0]);
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

// Shared-memory layout of the fused adjoint step.
template <class Real>
struct Adj2D {
  static constexpr int BX = 32, BY = 16, NT = BX * BY;  // threads: tile + one-cell halo
  static constexpr int OX = BX - 2, OY = BY - 2;        // output cells per CTA
  static constexpr int W2 = BX + 2, H2 = BY + 2, C2 = W2 * H2;  // tile + two-cell halo
  static constexpr int RING = 2 * W2 + 2 * BY;          // the outer ring of C2
  static constexpr int MIN_CTAS = sizeof(Real) == 4 ? 3 : 1;  // FP32: 40 registers, three CTAs per SM
  enum { S0, S1, MU0, AA, UX, UY, NCELL };              // per-cell values
  // per solute face: d/d mu_a, mu_b, s'_a, s'_b, U_a, U_b, s_a, s_b, and the
  // transverse antitrapping coefficient T (+T to a+t, b+t; -T to a-t, b-t)
  enum { F_MUA, F_MUB, F_SPA, F_SPB, F_UA, F_UB, F_SA, F_SB, F_T, NF };
  static constexpr size_t cell = 0;
  static constexpr size_t sface = cell + sizeof(Real) * NCELL * C2;  // [2][NF][C2] by a
  static constexpr size_t lu = sface + sizeof(Real) * 2 * NF * C2;   // [NT]
  static constexpr size_t mask = lu + sizeof(Real) * NT;             // [C2] bytes
  static constexpr size_t bytes = mask + ((C2 + 15) / 16) * 16;
  // the phase-field faces [2][cn, ct][NT] reuse the solute-face area
};

template <class Real>
__global__ void __launch_bounds__(Adj2D<Real>::NT, Adj2D<Real>::MIN_CTAS) adj2d_kernel(const DevParams<Real> P, const AdjIO<Real> io) {
  using S = Adj2D<Real>;
  using Lat = Lattice<9>;
  constexpr int BX = S::BX, BY = S::BY, NT = S::NT, W2 = S::W2, C2 = S::C2, NF = S::NF;
  extern __shared__ __align__(16) unsigned char smem[];
  Real* sc = reinterpret_cast<Real*>(smem + S::cell);
  Real* sf = reinterpret_cast<Real*>(smem + S::sface);
  Real* slu = reinterpret_cast<Real*>(smem + S::lu);
  Real* spf = sf;
  unsigned char* sm = smem + S::mask;

  const int nx = P.n[0], ny = P.n[1];
  const long long plane = P.plane;
  const int tid = threadIdx.x, tx = tid % BX, ty = tid / BX;
  const int x0 = blockIdx.x * S::OX, y0 = blockIdx.y * S::OY;
  const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;  // this thread's cell, unfolded
  // a tile whose two-cell halo lies inside the grid needs no folding
  const bool inner_tile = x0 >= 2 && x0 - 2 + W2 <= nx && y0 >= 2 && y0 - 2 + S::H2 <= ny;
  const int fx = inner_tile ? gx : fold_axis(P, gx, 0), fy = inner_tile ? gy : fold_axis(P, gy, 1);
  const long long o = (long long)fy * P.px + fx;
  const int h2 = (ty + 1) * W2 + tx + 1;  // this cell in the tile + two-cell halo
  const bool inner = tx >= 1 && tx <= BX - 2 && ty >= 1 && ty <= BY - 2 && gx < nx && gy < ny;
  const Real theta_base = Real(P.theta0) - Real(P.GV) * Real(io.clock[0]);
  const bool walls = (P.wall[0] | P.wall[1]) != 0;
  const Real e = P.inv2A[1] - P.inv2A[0];
  const Real mob = P.mob_eps * P.eps;  // 1 / tau_phi

  // Programmatic dependent launch: the next adjoint step may start as this
  // one's CTAs retire.  Until the wait below a step reads only the stored
  // forward states (written before the segment's adjoint began), never the
  // lambda of the previous step; everything it writes to global memory comes
  // after the wait, which returns once the previous step has finished and
  // its writes are visible.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  // 0. per-cell values: own cell, then the outer ring
  const Real s0 = __ldg(io.s0 + o), s1 = __ldg(io.s1 + o), mu0 = __ldg(io.mu0 + o);
  const bool obs = walls && obstacle(P, fx, fy, 0);
  Macro2<Real> m;
  Real Aown;
  {
    Real dk[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) dk[k] = __ldg(io.d0 + k * plane + o);
    m = macro2(P, dk, s0, mu0, obs, theta_base + P.G * Real(fy));
    sc[S::S0 * C2 + h2] = s0;
    sc[S::S1 * C2 + h2] = s1;
    sc[S::MU0 * C2 + h2] = mu0;
    sc[S::UX * C2 + h2] = m.ux;
    sc[S::UY * C2 + h2] = m.uy;
    sm[h2] = (unsigned char)((s0 > Real(0) ? 2u : 0u) | (Real(1) - s0 > Real(0) ? 1u : 0u) | (obs ? 4u : 0u));
  }
  long long q = 0;  // ring cell of threads tid < RING
  Real rden = Real(0);
  bool robs = false;
  int rc = 0;
  if (tid < S::RING) {
    int ri, rj;
    if (tid < W2) {
      ri = tid;
      rj = 0;
    } else if (tid < 2 * W2) {
      ri = tid - W2;
      rj = S::H2 - 1;
    } else if (tid < 2 * W2 + BY) {
      ri = 0;
      rj = tid - 2 * W2 + 1;
    } else {
      ri = W2 - 1;
      rj = tid - 2 * W2 - BY + 1;
    }
    const int qx = inner_tile ? x0 - 2 + ri : fold_axis(P, x0 - 2 + ri, 0);
    const int qy = inner_tile ? y0 - 2 + rj : fold_axis(P, y0 - 2 + rj, 1);
    q = (long long)qy * P.px + qx;
    const Real rs0 = __ldg(io.s0 + q), rs1 = __ldg(io.s1 + q), rmu = __ldg(io.mu0 + q);
    robs = walls && obstacle(P, qx, qy, 0);
    Real dk[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) dk[k] = __ldg(io.d0 + k * plane + q);
    const Macro2<Real> rm = macro2(P, dk, rs0, rmu, robs, theta_base + P.G * Real(qy));
    const int c = rj * W2 + ri;
    rc = c;
    rden = P.inv2A[0] + Hs(rs1) * e;
    sc[S::S0 * C2 + c] = rs0;
    sc[S::S1 * C2 + c] = rs1;
    sc[S::MU0 * C2 + c] = rmu;
    sc[S::UX * C2 + c] = rm.ux;
    sc[S::UY * C2 + c] = rm.uy;
    sm[c] = (unsigned char)((rs0 > Real(0) ? 2u : 0u) | (Real(1) - rs0 > Real(0) ? 1u : 0u) | (robs ? 4u : 0u));
  }
  // lambda^{n+1} is the previous step's output
  asm volatile("griddepcontrol.wait;" ::: "memory");
  Aown = obs ? Real(0) : io.lmu1[o] / (P.inv2A[0] + Hs(s1) * e);
  sc[S::AA * C2 + h2] = Aown;
  if (tid < S::RING) sc[S::AA * C2 + rc] = robs ? Real(0) : io.lmu1[q] / rden;
  __syncthreads();

  // 1. solute faces, by their lower cell a (tile + two-cell halo coordinates)
  auto solute_face = [&](int ia, int ja, int d) {
    Real cf[NF];
#pragma unroll
    for (int v = 0; v < NF; ++v) cf[v] = Real(0);
    const int ca = ja * W2 + ia, cb = ca + (d == 0 ? 1 : W2), st = d == 0 ? W2 : 1;
    const int gn = d == 0 ? x0 - 2 + ia : y0 - 2 + ja;  // a along the face normal
    const int gt = d == 0 ? y0 - 2 + ja : x0 - 2 + ia;  // a across it
    // the face exists only between two cells of the grid (walls do not wrap)
    bool closed = P.bc[d] == kWall && (gn < 0 || gn >= P.n[d] - 1);
    closed = closed || (P.bc[1 - d] == kWall && (gt < 0 || gt >= P.n[1 - d]));
    closed = closed || ((sm[ca] | sm[cb]) & 4u);  // no solute crosses obstacle faces
    if (!closed) {
      const Real s0a = sc[S::S0 * C2 + ca], s0b = sc[S::S0 * C2 + cb];
      const Real s1a = sc[S::S1 * C2 + ca], s1b = sc[S::S1 * C2 + cb];
      const Real mua = sc[S::MU0 * C2 + ca], mub = sc[S::MU0 * C2 + cb];
      const Real L = sc[S::AA * C2 + cb] - sc[S::AA * C2 + ca];  // adjoint of the face flux
      const Real ua = sc[(d == 0 ? S::UX : S::UY) * C2 + ca], ub = sc[(d == 0 ? S::UX : S::UY) * C2 + cb];
      // diffusion -M_f (mu_b - mu_a), M = M0 (1 - s')
      const Real Mf = Real(0.5) * P.M0 * ((Real(1) - s1a) + (Real(1) - s1b));
      const Real dM = L * Real(0.5) * P.M0 * (mub - mua);
      cf[S::F_MUA] = L * Mf;
      cf[S::F_MUB] = -L * Mf;
      cf[S::F_SPA] = dM;
      cf[S::F_SPB] = dM;
      // advection 1/2 [U_d h0' c0(mu)]_a + [..]_b with h0' = 1 - H(s')
      const Real h0a = Real(1) - Hs(s1a), h0b = Real(1) - Hs(s1b);
      // T - T_E of cells a and b (vertical index folded as the loads were),
      // needed only when ceq depends on T
      Real tha = Real(0), thb = Real(0);
      if (P.tdep) {
        const int ya = inner_tile ? y0 - 2 + ja : fold_axis(P, y0 - 2 + ja, 1);
        const int yb = d == 1 ? (inner_tile ? ya + 1 : fold_axis(P, y0 - 1 + ja, 1)) : ya;
        tha = theta_base + P.G * Real(ya);
        thb = theta_base + P.G * Real(yb);
      }
      const Real c0a = P.ceq[0][0] + P.dceq_dT[0][0] * tha + mua * P.inv2A[0];
      const Real c0b = P.ceq[0][0] + P.dceq_dT[0][0] * thb + mub * P.inv2A[0];
      cf[S::F_UA] = L * Real(0.5) * h0a * c0a;
      cf[S::F_UB] = L * Real(0.5) * h0b * c0b;
      cf[S::F_MUA] += L * Real(0.5) * ua * h0a * P.inv2A[0];
      cf[S::F_MUB] += L * Real(0.5) * ub * h0b * P.inv2A[0];
      cf[S::F_SPA] -= L * Real(0.5) * ua * c0a * dHs(s1a);
      cf[S::F_SPB] -= L * Real(0.5) * ub * c0b * dHs(s1b);
      // antitrapping -a eps liq dc dphi n_d (liq, n at time n)
      if (P.at_eps != Real(0)) {
        const Real g_n = s0b - s0a;
        const Real g_t = Real(0.25) * (sc[S::S0 * C2 + ca + st] + sc[S::S0 * C2 + cb + st] -
                                       sc[S::S0 * C2 + ca - st] - sc[S::S0 * C2 + cb - st]);
        const Real g2 = g_n * g_n + g_t * g_t;
        if (g2 > Real(1e-12)) {
          const Real rg = Real(1) / sqrt(g2);
          const Real nd = g_n * rg;
          const Real liq = Real(1) - Real(0.5) * (s0a + s0b);
          const Real dinv = P.inv2A[0] - P.inv2A[1];
          const Real dc = (P.ceq[0][0] - P.ceq[1][0]) +
                          (P.dceq_dT[0][0] - P.dceq_dT[1][0]) * Real(0.5) * (tha + thb) +
                          Real(0.5) * (mua + mub) * dinv;
          const Real dphi = Real(0.5) * ((s1a - s0a) + (s1b - s0b));
          const Real k = -P.at_eps * L;
          const Real jl = k * dc * dphi * nd;   // d / d liq
          const Real jc = k * liq * dphi * nd;  // d / d dc
          const Real jp = k * liq * dc * nd;    // d / d dphi
          const Real jn = k * liq * dc * dphi;  // d / d n_d
          const Real r3 = rg * rg * rg;
          const Real dn_n = g_t * g_t * r3, dn_t = -g_n * g_t * r3;
          cf[S::F_SA] += -Real(0.5) * jl - Real(0.5) * jp - jn * dn_n;
          cf[S::F_SB] += -Real(0.5) * jl - Real(0.5) * jp + jn * dn_n;
          cf[S::F_SPA] += Real(0.5) * jp;
          cf[S::F_SPB] += Real(0.5) * jp;
          cf[S::F_MUA] += Real(0.5) * dinv * jc;
          cf[S::F_MUB] += Real(0.5) * dinv * jc;
          cf[S::F_T] = Real(0.25) * jn * dn_t;
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NF; ++v) sf[(d * NF + v) * C2 + ca] = cf[v];
  };
  solute_face(tx + 1, ty + 1, 0);
  solute_face(tx + 1, ty + 1, 1);
  // the faces below the one-cell halo: a in the left column / bottom row
  if (tid < BY) solute_face(0, tid + 1, 0);
  else if (tid >= 32 && tid < 32 + BX) solute_face(tid - 32 + 1, 0, 1);
  __syncthreads();

  // 2. lambda through the mu stage, the faces and the collision
  auto F = [&](int d, int v, int c) { return sf[(d * NF + v) * C2 + c]; };
  Real lsp = io.ls1[o] + F(0, S::F_SPA, h2) + F(1, S::F_SPA, h2) + F(0, S::F_SPB, h2 - 1) +
             F(1, S::F_SPB, h2 - W2);
  Real lmu = io.lmu1[o];
  Real ls = Real(0);
  const Real mu1 = __ldg(io.mu1 + o);
  if (!obs) {
    // mu' = mu + (-div J - src) / chi', src = (c1 - c0)(mu, T) (H(s') - H(s))
    //   - (dT/dt) (dceq_0/dT (1 - H(s')) + dceq_1/dT H(s')),  dT/dt = -G V
    const Real th = theta_base + P.G * Real(fy);
    const Real c10 = (P.ceq[1][0] - P.ceq[0][0]) + (P.dceq_dT[1][0] - P.dceq_dT[0][0]) * th + mu0 * e;
    lmu -= Aown * e * (Hs(s1) - Hs(s0));
    lsp += -Aown * c10 * dHs(s1) - Aown * (mu1 - mu0) * e * dHs(s1);
    lsp += Aown * Real(P.GV) * (P.dceq_dT[1][0] - P.dceq_dT[0][0]) * dHs(s1);
    ls += Aown * c10 * dHs(s0);
  }
  bool multi = false;
  if (!obs) {
    unsigned act = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) act |= sm[h2 + dy * W2 + dx];
    multi = (act & 3u) == 3u;
  }
  const Real lu = (multi && s1 > Real(0) && s1 < Real(1)) ? lsp : Real(0);
  slu[tid] = lu;

  if (inner) {
    lmu += F(0, S::F_MUA, h2) + F(1, S::F_MUA, h2) + F(0, S::F_MUB, h2 - 1) + F(1, S::F_MUB, h2 - W2);
    ls += F(0, S::F_SA, h2) + F(1, S::F_SA, h2) + F(0, S::F_SB, h2 - 1) + F(1, S::F_SB, h2 - W2);
    // antitrapping across x-faces (transverse y) and y-faces (transverse x)
    ls += F(0, S::F_T, h2 - W2) + F(0, S::F_T, h2 - W2 - 1) - F(0, S::F_T, h2 + W2) - F(0, S::F_T, h2 + W2 - 1);
    ls += F(1, S::F_T, h2 - 1) + F(1, S::F_T, h2 - 1 - W2) - F(1, S::F_T, h2 + 1) - F(1, S::F_T, h2 + 1 - W2);
    if (P.bc[1] == kWall) {  // the wall mirrors a-t / a+t onto the row next to it
      if (gy == 0) ls -= F(0, S::F_T, h2) + F(0, S::F_T, h2 - 1);
      if (gy == ny - 1) ls += F(0, S::F_T, h2) + F(0, S::F_T, h2 - 1);
    }
    if (P.bc[0] == kWall) {
      if (gx == 0) ls -= F(1, S::F_T, h2) + F(1, S::F_T, h2 - W2);
      if (gx == nx - 1) ls += F(1, S::F_T, h2) + F(1, S::F_T, h2 - W2);
    }
    Real gUx = F(0, S::F_UA, h2) + F(0, S::F_UB, h2 - 1);
    Real gUy = F(1, S::F_UA, h2) + F(1, S::F_UB, h2 - W2);

    // populations: pull transposed (bounce-back at walls), then BGK + Guo
    Real a[9];
    if (fx >= 1 && fx <= nx - 2 && fy >= 1 && fy <= ny - 2) {  // no wall or wrap in reach
#pragma unroll
      for (int k = 0; k < 9; ++k) a[k] = io.ld1[k * plane + o + Lat::c(k, 0) + Lat::c(k, 1) * P.px];
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        int qx = fx + Lat::c(k, 0), qy = fy + Lat::c(k, 1);
        const bool bounce = (P.bc[0] == kWall && (qx < 0 || qx >= nx)) || (P.bc[1] == kWall && (qy < 0 || qy >= ny));
        if (bounce) {
          a[k] = io.ld1[Lat::opp(k) * plane + o];
        } else {
          qx = qx < 0 ? qx + nx : (qx >= nx ? qx - nx : qx);
          qy = qy < 0 ? qy + ny : (qy >= ny ? qy - ny : qy);
          a[k] = io.ld1[k * plane + (long long)qy * P.px + qx];
        }
      }
    }
    // f*_k = omega d_k + (feq_k - w_k) / tau + G_k is a quadratic in U and
    // linear in F and rho, so its transpose needs only the moments of
    // a_k w_k: S0 = sum, S1 = sum c_k, S2 = sum c_k c_k.
    Real S0 = Real(0), S1x = Real(0), S1y = Real(0), Sxx = Real(0), Sxy = Real(0), Syy = Real(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const Real aw = a[k] * Real(Lat::w(k));
      const int cx = Lat::c(k, 0), cy = Lat::c(k, 1);
      S0 += aw;
      if (cx) S1x += cx > 0 ? aw : -aw;
      if (cy) S1y += cy > 0 ? aw : -aw;
      if (cx) Sxx += aw;
      if (cy) Syy += aw;
      if (cx && cy) Sxy += cx * cy > 0 ? aw : -aw;
    }
    const Real omega = Real(1) - P.inv_tau_f, pre = P.force_pre, itau = P.inv_tau_f;
    const Real uu = m.ux * m.ux + m.uy * m.uy;
    const Real SUx = Sxx * m.ux + Sxy * m.uy, SUy = Sxy * m.ux + Syy * m.uy;  // S2 U
    const Real SFx = Sxx * m.Fx + Sxy * m.Fy, SFy = Sxy * m.Fx + Syy * m.Fy;  // S2 F
    // V = -3 U S0 + 3 S1 + 9 S2 U: d/dF = pre V, d/dU = rho V / tau - 3 pre F S0 + 9 pre S2 F
    const Real Vx = Real(-3) * m.ux * S0 + Real(3) * S1x + Real(9) * SUx;
    const Real Vy = Real(-3) * m.uy * S0 + Real(3) * S1y + Real(9) * SUy;
    Real gr = itau * (S0 * (Real(1) - Real(1.5) * uu) + Real(3) * (m.ux * S1x + m.uy * S1y) +
                      Real(4.5) * (m.ux * SUx + m.uy * SUy));
    gUx += itau * m.rho * Vx + pre * (Real(-3) * m.Fx * S0 + Real(9) * SFx);
    gUy += itau * m.rho * Vy + pre * (Real(-3) * m.Fy * S0 + Real(9) * SFy);
    const Real gFx = pre * Vx, gFy = pre * Vy;
    // F = F_B e_y - rho kappa U;  U = (m + F_B/2 e_y) iv;  iv = 1/(rho (1 + kappa/2))
    gUx += -m.rho * m.kappa * gFx;
    gUy += -m.rho * m.kappa * gFy;
    gr += -m.kappa * (m.ux * gFx + m.uy * gFy);
    Real gk = -m.rho * (m.ux * gFx + m.uy * gFy);
    Real gFB = gFy + Real(0.5) * gUy * m.iv;
    const Real gmx = gUx * m.iv, gmy = gUy * m.iv;
    const Real giv = gUx * m.mx + gUy * (m.my + Real(0.5) * m.FB);
    gr += giv * (-m.iv / m.rho);
    gk += giv * (-Real(0.5) * m.rho * m.iv * m.iv);
    gr += gFB * m.phil * m.B;  // F_B = rho phil B
    const Real gphil = gFB * m.rho * m.B + gk * (-Real(2) * P.kappa0 * (Real(1) - m.phil));
    const Real gB = gFB * m.rho * m.phil;
#pragma unroll
    for (int k = 0; k < 9; ++k)
      io.ld0[k * plane + o] = omega * a[k] + gr + Real(Lat::c(k, 0)) * gmx + Real(Lat::c(k, 1)) * gmy;
    if (!obs) ls -= gphil;  // phil = 1 - s
    lmu += gB * P.gbeta_c[0] * P.inv2A[0];
    io.gacc[2 * plane + o] +=
        (double)(gB * (P.dcl_ref[0] + P.dceq_dT[0][0] * (theta_base + P.G * Real(fy)) + mu0 * P.inv2A[0]));

    // phase field: s' = clamp(u) where both phases are present, s' = s elsewhere
    if (multi) {
      if (lu != Real(0)) {
        const Real thc = theta_base + P.G * Real(fy);
        const Real dceq = (P.ceq[1][0] - P.ceq[0][0]) + (P.dceq_dT[1][0] - P.dceq_dT[0][0]) * thc;
        const Real dpsi = -mu0 * mu0 * (P.inv4A[1] - P.inv4A[0]) - mu0 * dceq + (P.S[1] - P.S[0]) * thc;
        const Real dpsi_dmu = -mu0 * e - dceq;
        const Real cob = P.obst * P.gamma[0][1] / P.eps;  // 16 gamma / (pi^2 eps^2)
        ls += lu * (Real(1) + Real(0.5) * mob * (Real(2) * cob - (Real(6) / P.eps) * (Real(1) - Real(2) * s0) * dpsi));
        lmu += lu * Real(0.5) * mob * (-(Real(6) / P.eps) * s0 * (Real(1) - s0) * dpsi_dmu);
        io.gacc[0 * plane + o] += (double)(lu * (s1 - s0) / mob);
      }
    } else {
      ls += lsp;
    }
    io.lmu0[o] = lmu;
  }
  __syncthreads();

  // 3. phase-field faces: lambda_V = (mob/2) gamma (lu(a) - lu(b)) through
  //    V_d = dA/dq_d(grad_f s) to the six cells of the face stencil
  {
    const Real gam = P.gamma[0][1];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      Real cn = Real(0), ct = Real(0);
      const bool has = d == 0 ? tx <= BX - 2 : ty <= BY - 2;  // b inside the one-cell halo
      const int gn = d == 0 ? gx : gy, gt = d == 0 ? gy : gx;
      const bool closed = (P.bc[d] == kWall && (gn < 0 || gn >= P.n[d] - 1)) ||
                          (P.bc[1 - d] == kWall && (gt < 0 || gt >= P.n[1 - d]));
      if (has && !closed) {
        const Real lV = Real(0.5) * mob * gam * (lu - slu[tid + (d == 0 ? 1 : BX)]);
        if (lV != Real(0)) {
          const int ca = h2, cb = h2 + (d == 0 ? 1 : W2), st = d == 0 ? W2 : 1;
          const Real g_n = sc[S::S0 * C2 + cb] - sc[S::S0 * C2 + ca];
          const Real g_t = Real(0.25) * (sc[S::S0 * C2 + ca + st] + sc[S::S0 * C2 + cb + st] -
                                         sc[S::S0 * C2 + ca - st] - sc[S::S0 * C2 + cb - st]);
          Real dV[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            Tan<Real> q[2];
            q[d] = Tan<Real>(g_n, j == 0 ? Real(1) : Real(0));
            q[1 - d] = Tan<Real>(g_t, j == 1 ? Real(1) : Real(0));
            const Tan<Real> dl(P.delta[0][1], j == 2 ? Real(1) : Real(0));
            dV[j] = P.tilted ? dAdq_tan_tilted<Real>(q, dl, P.tilt_c[0][1], P.tilt_s[0][1], P.q_floor, d).d
                             : dAdq_tan<Real>(q, dl, P.q_floor, d).d;
          }
          cn = lV * dV[0];
          ct = Real(0.25) * lV * dV[1];
          if (inner) io.gacc[1 * plane + o] += (double)(lV * dV[2]);
        }
      }
      spf[(d * 2 + 0) * NT + tid] = cn;
      spf[(d * 2 + 1) * NT + tid] = ct;
    }
  }
  __syncthreads();
  if (inner) {
    auto CN = [&](int d, int t) { return spf[(d * 2 + 0) * NT + t]; };
    auto CT = [&](int d, int t) { return spf[(d * 2 + 1) * NT + t]; };
    ls += CN(0, tid - 1) - CN(0, tid) + CN(1, tid - BX) - CN(1, tid);
    ls += CT(0, tid - BX) + CT(0, tid - BX - 1) - CT(0, tid + BX) - CT(0, tid + BX - 1);
    ls += CT(1, tid - 1) + CT(1, tid - 1 - BX) - CT(1, tid + 1) - CT(1, tid + 1 - BX);
    if (P.bc[1] == kWall) {
      if (gy == 0) ls -= CT(0, tid) + CT(0, tid - 1);
      if (gy == ny - 1) ls += CT(0, tid) + CT(0, tid - 1);
    }
    if (P.bc[0] == kWall) {
      if (gx == 0) ls -= CT(1, tid) + CT(1, tid - BX);
      if (gx == nx - 1) ls += CT(1, tid) + CT(1, tid - BX);
    }
    io.ls0[o] = ls;
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
    acc += Hs((double)s[off2(P, x, y)]);  // J in FP64 from the stored state
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

// One plane from the exchange layout into the internal layout.
template <class Real>
__global__ void adj_import_kernel(const DevParams<Real> P, const Real* __restrict__ src, Real* __restrict__ dst) {
  const long long cells = (long long)P.n[0] * P.n[1];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= cells) return;
  int x, y;
  cell_xy(P, c, &x, &y);
  dst[off2(P, x, y)] = src[c];
}

}  // namespace gpflbm

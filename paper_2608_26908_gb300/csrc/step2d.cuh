// Fused 2D step kernel for sm_103a: one launch advances the grid by one time
// step (Algorithm 1: phase field, chemical potential, lattice Boltzmann).
//
// A CTA owns a tile and runs one thread per cell of the tile's one-cell halo
// region ("R1", BX x BY cells); the (BX-2) x (BY-2) inner cells are written.
// Every shared-memory access of a thread is at a fixed offset from its own
// cell, so there is no per-access index arithmetic.  Per CTA:
//   0. each thread loads its cell (phi^n, mu^n, f^n), and the threads of the
//      first warps also the ring of cells around R1 (phi^n only, for the
//      phase-field stencil); it collides its own populations (BGK + Guo
//      forcing with the implicit drag velocity and buoyancy) into shared
//      memory and records which phases are present;
//   1. where more than one phase is present in a 3x3 neighbourhood, the
//      phase-field face fluxes and the update of Eq. PhfGrand (obstacle
//      potential, Lambda over the present phases, Gibbs-simplex projection);
//      elsewhere phi^{n+1} = phi^n exactly (the one present phase has rate 0);
//   2. the solute flux through each cell's +x and +y face (diffusion,
//      antitrapping, advection by U^n);
//   3. inner cells: mu^{n+1}, phi^{n+1}, and f^{n+1} pulled from the collided
//      populations of the neighbours (halfway bounce-back on walls).
// A face flux of the phase field is exactly zero when the six cells it reads
// hold one pure phase, so each face is evaluated only where its cells mix.
#pragma once

#include "gpflbm_kernels.cuh"

namespace gpflbm {

template <class Real>
struct Block2D;
// MIN_CTAS: resident CTAs per SM the register budget is cut for (FP32: three,
// 40 registers a thread, 48 warps; FP64: four CTAs of 256 threads, 64
// registers).
template <>
struct Block2D<float> {
  static constexpr int BX = 32, BY = 16, MIN_CTAS = 3;
};
template <>
struct Block2D<double> {
  // half-height tiles: FP64 arithmetic is slow on this part, and the small
  // FP64 grids need the CTAs spread over every SM
  static constexpr int BX = 32, BY = 8, MIN_CTAS = 4;
};

template <int NP, int NC, class Real, class Store>
struct Step2D {
  static constexpr int BX = Block2D<Real>::BX, BY = Block2D<Real>::BY;
  static constexpr int NT = BX * BY, Q = 9;
  static constexpr int OX = BX - 2, OY = BY - 2;                // inner (output) cells
  static constexpr int W2 = BX + 2, H2 = BY + 2, C2 = W2 * H2;  // R1 plus one ring
  static constexpr int RING = C2 - NT;
  static constexpr int PFX = (BX + 1) * BY, PFY = BX * (BY + 1);  // phase-field faces of R1
  static constexpr size_t al(size_t v) { return (v + 15) / 16 * 16; }
  static constexpr size_t phi = 0;                                  // NP x C2
  static constexpr size_t fs = al(phi + sizeof(Real) * NP * C2);    // Q x NT (collided)
  static constexpr size_t u = al(fs + sizeof(Store) * Q * NT);      // 2 x NT
  static constexpr size_t mu = al(u + sizeof(Real) * 2 * NT);       // NC x NT
  static constexpr size_t pn = al(mu + sizeof(Real) * NC * NT);     // NP x NT
  static constexpr size_t hl = al(pn + sizeof(Real) * NP * NT);     // NT
  static constexpr size_t flux = al(hl + sizeof(Real) * NT);        // PF or solute faces
  static constexpr size_t flux_n =
      NP * (PFX + PFY) > 2 * NC * NT ? NP * (PFX + PFY) : 2 * NC * NT;
  static constexpr size_t mask = al(flux + sizeof(Real) * flux_n);  // C2 bytes
  static constexpr size_t chg = al(mask + C2);                      // NT bytes
  static constexpr size_t bytes = al(chg + NT);
};

struct Step2DIO {
  const void* phi_in;
  void* phi_out;
  const void* mu_in;
  void* mu_out;
  const void* f_in;
  void* f_out;
  const double* clock_in;
  double* clock_out;
};

// EXT: the extended model -- pairs' crystal axes turned about z (dAdq_pair)
// and equilibrium compositions ceq_a(T) with the temperature term of Eq. conc.
// SHRINK: the shrinkage force needs phi^{n+1}, so the collision moves after
// the phase-field update (the raw populations wait in the collision buffer).
template <int NP, int NC, class Real, class Store, bool SHRINK = false, bool EXT = false>
__global__ void __launch_bounds__(Step2D<NP, NC, Real, Store>::NT, Block2D<Real>::MIN_CTAS)
    step2d_kernel(const DevParams<Real> P, const Step2DIO io) {
  using S = Step2D<NP, NC, Real, Store>;
  using Lat = Lattice<9>;
  constexpr int BX = S::BX, BY = S::BY, NT = S::NT, Q = 9, W2 = S::W2, H2 = S::H2, C2 = S::C2;
  constexpr int NS = PhiStore<NP>::NS;
  extern __shared__ __align__(16) unsigned char smem[];
  Real* s_phi = reinterpret_cast<Real*>(smem + S::phi);
  Store* s_fs = reinterpret_cast<Store*>(smem + S::fs);
  Real* s_u = reinterpret_cast<Real*>(smem + S::u);
  Real* s_mu = reinterpret_cast<Real*>(smem + S::mu);
  Real* s_pn = reinterpret_cast<Real*>(smem + S::pn);
  Real* s_hl = reinterpret_cast<Real*>(smem + S::hl);
  Real* s_flux = reinterpret_cast<Real*>(smem + S::flux);
  unsigned char* s_mask = smem + S::mask;
  unsigned char* s_chg = smem + S::chg;

  const Real* __restrict__ phi_in = static_cast<const Real*>(io.phi_in);
  const Real* __restrict__ mu_in = static_cast<const Real*>(io.mu_in);
  const Store* __restrict__ f_in = static_cast<const Store*>(io.f_in);

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int nx = P.n[0], ny = P.n[1], px = P.px;
  const int x0 = blockIdx.x * S::OX, y0 = blockIdx.y * S::OY;  // first inner cell
  const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;                 // this thread's cell
  const bool inner_tile = x0 >= 2 && x0 - 2 + W2 <= nx && y0 >= 2 && y0 - 2 + H2 <= ny;
  const int fx = inner_tile ? gx : fold_axis(P, gx, 0);
  const int fy = inner_tile ? gy : fold_axis(P, gy, 1);
  const int g = fy * px + fx;  // a plane holds fewer than 2^31 cells
  const int r2 = (ty + 1) * W2 + tx + 1;  // this cell in the R1-plus-ring layout
  const double t_now = io.clock_in[0];
  if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) io.clock_out[0] = t_now + 1.0;
  const Real theta_base = Real(P.theta0) - Real(P.GV) * Real(t_now);
  const bool obs = (P.wall[0] | P.wall[1]) != 0 && obstacle(P, fx, fy, 0);
  // EXT: ceq_a,i(T) of this cell, T - T_E = theta_base + G v
  auto ceq_of = [&](int a, int i, int v) -> Real {
    if constexpr (EXT)
      return P.ceq[a][i] + P.dceq_dT[a][i] * (theta_base + P.G * Real(v));
    else
      return P.ceq[a][i];
  };

  // 0. own cell: phases present, mu; ring cells (phi only); collision
  // a cell of pure liquid: phi_0 = 1 and every other phase 0, exactly
  auto pure_liquid = [](const Real* v) {
    bool p = v[0] == Real(1);
#pragma unroll
    for (int a = 1; a < NP; ++a) p = p && v[a] == Real(0);
    return p;
  };
  Real ph[NP];
  load_phases<NP>(phi_in, g, P.plane, ph);
  bool liquid = pure_liquid(ph) && !obs;  // the tile's cells, for the liquid-tile path
  // the ring cell of a thread tid < RING: its R1-plus-ring index rr and its
  // offset in a plane
  auto ring_cell = [&](int& rr) {
    int rx, ry;
    if (tid < W2) {
      rx = tid;
      ry = 0;
    } else if (tid < 2 * W2) {
      rx = tid - W2;
      ry = H2 - 1;
    } else if (tid < 2 * W2 + H2 - 2) {
      rx = 0;
      ry = tid - 2 * W2 + 1;
    } else {
      rx = W2 - 1;
      ry = tid - 2 * W2 - (H2 - 2) + 1;
    }
    const int qx = inner_tile ? x0 - 2 + rx : fold_axis(P, x0 - 2 + rx, 0);
    const int qy = inner_tile ? y0 - 2 + ry : fold_axis(P, y0 - 2 + ry, 1);
    rr = ry * W2 + rx;
    return qy * px + qx;
  };
  if (tid < S::RING) {
    int rr;
    Real rv[NP];
    load_phases<NP>(phi_in, ring_cell(rr), P.plane, rv);
    liquid = liquid && pure_liquid(rv);
  }
  // phi^n and the phases present, in shared memory for the phase-field
  // stencil (the general path only; the ring is read again here rather than
  // held in registers through the collision)
  auto stage_phi = [&]() {
    unsigned m = 0;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      s_phi[a * C2 + r2] = ph[a];
      if (ph[a] > Real(0)) m |= 1u << a;
    }
    s_mask[r2] = (unsigned char)m;
    if (tid < S::RING) {
      int rr;
      Real rv[NP];
      load_phases<NP>(phi_in, ring_cell(rr), P.plane, rv);
      m = 0;
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        s_phi[a * C2 + rr] = rv[a];
        if (rv[a] > Real(0)) m |= 1u << a;
      }
      s_mask[rr] = (unsigned char)m;
    }
  };
  Real mu[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    mu[i] = (mu_in + i * P.plane)[g];
    s_mu[i * NT + tid] = mu[i];
  }
  // moments, U, F (drag, buoyancy and, with SHRINK, the shrinkage force fs)
  // and the collision of this cell's populations into shared memory
  auto lbm_cell = [&](const Real* dk, Real fsx, Real fsy) {
    const Real drho = ((dk[0] + dk[1]) + (dk[2] + dk[3])) + ((dk[4] + dk[5]) + (dk[6] + dk[7])) + dk[8];
    const Real mx = (dk[1] - dk[3]) + (dk[5] - dk[6]) + (dk[8] - dk[7]);
    const Real my = (dk[2] - dk[4]) + (dk[5] + dk[6]) - (dk[7] + dk[8]);
    const Real rho = Real(1) + drho;
    const Real phil = obs ? Real(0) : ph[0];
    const Real sl = Real(1) - phil;
    const Real kappa = P.kappa0 * sl * sl;
    Real drive = P.gbeta_T * (theta_base + P.G * Real(fy) + P.dT_ref);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      if constexpr (EXT)
        drive += P.gbeta_c[i] * (P.dcl_ref[i] + P.dceq_dT[0][i] * (theta_base + P.G * Real(fy)) +
                                 mu[i] * P.inv2A[0]);
      else
        drive += P.gbeta_c[i] * (P.dcl_ref[i] + mu[i] * P.inv2A[0]);
    }
    const Real FB = rho * phil * drive;
    const Real inv = rcp_rn(rho * (Real(1) + Real(0.5) * kappa));
    Real ux, uy, Fx, Fy;
    if constexpr (SHRINK) {
      ux = (mx + Real(0.5) * fsx) * inv;
      uy = (my + Real(0.5) * (FB + fsy)) * inv;
      Fx = fsx - rho * kappa * ux;
      Fy = FB + fsy - rho * kappa * uy;
    } else {
      ux = mx * inv;
      uy = (my + Real(0.5) * FB) * inv;
      Fx = -rho * kappa * ux;
      Fy = FB - rho * kappa * uy;
    }
    s_u[tid] = ux;
    s_u[NT + tid] = uy;
    const Real uv2[2] = {ux, uy}, Fv2[2] = {Fx, Fy};
    collide<Q>(P, dk, drho, rho, uv2, Fv2,
               [&](int k, Real val) { s_fs[k * NT + tid] = Codec<Store>::put(val); });
  };
  {
    Real dk[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) dk[k] = Codec<Store>::load(at_bytes(f_in + g, P.f_at[k]));
    if constexpr (SHRINK) {
#pragma unroll
      for (int k = 0; k < Q; ++k) s_fs[k * NT + tid] = Codec<Store>::put(dk[k]);  // exact round trip
    } else {
      lbm_cell(dk, Real(0), Real(0));
    }
  }
  // the inner cells write mu^{n+1}, phi^{n+1} and pull f^{n+1}
  const bool inner = !(tx < 1 || tx > BX - 2 || ty < 1 || ty > BY - 2 || gx >= nx || gy >= ny);
  Real* __restrict__ phi_out = static_cast<Real*>(io.phi_out);
  Real* __restrict__ mu_out = static_cast<Real*>(io.mu_out);
  Store* __restrict__ f_out = static_cast<Store*>(io.f_out);
  auto pull_f = [&]() {
    if (inner_tile) {
#pragma unroll
      for (int k = 0; k < Q; ++k)
        at_bytes(f_out + g, P.f_at[k]) = s_fs[k * NT + tid - Lat::c(k, 0) - Lat::c(k, 1) * BX];
    } else {
      const bool wx = P.bc[0] == kWall, wy = P.bc[1] == kWall;
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const int cx = Lat::c(k, 0), cy = Lat::c(k, 1);
        const bool bounce =
            (wx && (gx - cx < 0 || gx - cx >= nx)) || (wy && (gy - cy < 0 || gy - cy >= ny));
        const Store v = bounce ? s_fs[Lat::opp(k) * NT + tid] : s_fs[k * NT + tid - cx - cy * BX];
        at_bytes(f_out + g, P.f_at[k]) = v;
      }
    }
  };

  // Liquid tile: every cell of R1 and its ring is pure liquid and none is an
  // obstacle.  The phase field stays exactly as it is, h_l = 1, M = M0,
  // chi = 1 / (2 A_l) and there is no antitrapping, so the general path
  // below reduces to these few lines (the same arithmetic, term for term).
  if (__syncthreads_and(liquid)) {
    if constexpr (SHRINK) {
      // F_S = 0 where nothing solidifies: the deferred collision of the
      // general path with a zero shrinkage force
      Real dk[Q];
#pragma unroll
      for (int k = 0; k < Q; ++k) dk[k] = Codec<Store>::load(s_fs[k * NT + tid]);
      lbm_cell(dk, Real(0), Real(0));
      __syncthreads();
    }
    auto face = [&](int d) {
      const int nb = d == 0 ? tid + 1 : tid + BX;
      const int gbd = (d == 0 ? gx : gy) + 1;
      const bool closed = (P.bc[d] == kWall && (gbd == 0 || gbd == P.n[d])) || gbd > P.n[d];
      Real J[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) J[i] = Real(0);
      if (!closed) {
        const Real Mf = P.M0;                                   // 0.5 M0 (1 + 1)
        const Real ua = s_u[d * NT + tid], ub = s_u[d * NT + nb];  // h_l = 1
        const int vb = d == 0 ? fy : (inner_tile ? fy + 1 : fold_axis(P, gy + 1, 1));
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          const Real ma = s_mu[i * NT + tid], mb = s_mu[i * NT + nb];
          J[i] = -Mf * (mb - ma) + Real(0.5) * (ua * (ceq_of(0, i, fy) + ma * P.inv2A[0]) +
                                                ub * (ceq_of(0, i, vb) + mb * P.inv2A[0]));
        }
      }
#pragma unroll
      for (int i = 0; i < NC; ++i) s_flux[i * 2 * NT + d * NT + tid] = J[i];
    };
    if (tx < BX - 1) face(0);
    if (ty < BY - 1) face(1);
    __syncthreads();
    if (!inner) return;
#pragma unroll
    for (int sidx = 0; sidx < NS; ++sidx) (phi_out + sidx * P.plane)[g] = ph[NP == 2 ? 1 : sidx];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const Real* Ji = s_flux + i * 2 * NT;
      const Real div = (Ji[tid] - Ji[tid - 1]) + (Ji[NT + tid] - Ji[NT + tid - BX]);
      Real src = Real(0);
      if constexpr (EXT) {
#pragma unroll
        for (int a = 0; a < NP; ++a) src -= Real(P.GV) * P.dceq_dT[a][i] * (a == 0 ? Real(1) : Real(0));
      }
      (mu_out + i * P.plane)[g] = mu[i] + (-div - src) * P.chi_pure[0];
    }
    pull_f();
    return;
  }

  stage_phi();
  __syncthreads();

  // 1. phase field where phases mix
  unsigned act = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) act |= s_mask[r2 + dy * W2 + dx];
  const bool multi = __popc(act) >= 2 && !obs;
  Real out[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) out[a] = ph[a];
  if (__syncthreads_or(multi)) {
    // face fluxes -sum_{b != a} gamma_ab phi_b dA/dq(q_ab) on the +x / +y face
    // of this cell, and on the -x / -y face for the first column / row
    auto pf_face = [&](int ca, int cb, int d, int gbd, int slot) {
      // ca, cb: R1-plus-ring indices of the two cells; d: normal axis;
      // gbd: global index of the upper cell along d
      const int st = d == 0 ? W2 : 1;  // transverse stride
      const unsigned grp = s_mask[ca] | s_mask[cb] | s_mask[ca + st] | s_mask[cb + st] |
                           s_mask[ca - st] | s_mask[cb - st];
      const bool closed = P.bc[d] == kWall && (gbd == 0 || gbd == P.n[d]);
      Real fl[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) fl[a] = Real(0);
      if (__popc(grp) >= 2 && !closed) {
        Real pf[NP], gn[NP], gt[NP];
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          const Real* sp = s_phi + a * C2;
          pf[a] = Real(0.5) * (sp[ca] + sp[cb]);
          gn[a] = sp[cb] - sp[ca];
          // dA/dq = 2 q without anisotropy: only q_d enters the flux
          gt[a] = P.aniso ? Real(0.25) * (sp[ca + st] + sp[cb + st] - sp[ca - st] - sp[cb - st]) : Real(0);
        }
#pragma unroll
        for (int a = 0; a < NP; ++a)
#pragma unroll
          for (int b = a + 1; b < NP; ++b) {
            // a pair with a phase absent from the stencil has q = 0: exactly 0
            const Real gab = P.gamma[a][b];
            if (gab == Real(0) || (grp & ((1u << a) | (1u << b))) != ((1u << a) | (1u << b))) continue;
            Real q[2];
            q[d] = pf[a] * gn[b] - pf[b] * gn[a];
            q[1 - d] = pf[a] * gt[b] - pf[b] * gt[a];
            const Real v = dAdq_pair<2, EXT>(P, a, b, q, d);
            fl[a] -= gab * pf[b] * v;  // dA/dq(q_ba) = -dA/dq(q_ab)
            fl[b] += gab * pf[a] * v;
          }
      }
#pragma unroll
      for (int a = 0; a < NP; ++a) s_flux[a * (S::PFX + S::PFY) + slot] = fl[a];
    };
    // x-face i (between R1 columns i-1 and i) of row ty sits at slot ty*(BX+1)+i
    pf_face(r2, r2 + 1, 0, gx + 1, ty * (BX + 1) + tx + 1);
    if (tx == 0) pf_face(r2 - 1, r2, 0, gx, ty * (BX + 1));
    // y-face j (between R1 rows j-1 and j) of column tx sits at slot PFX + j*BX + tx
    pf_face(r2, r2 + W2, 1, gy + 1, S::PFX + (ty + 1) * BX + tx);
    if (ty == 0) pf_face(r2 - W2, r2, 1, gy, S::PFX + tx);
    __syncthreads();
    if (multi) {
      Real div[NP], gc[NP][2];
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        const Real* fa = s_flux + a * (S::PFX + S::PFY);
        div[a] = (fa[ty * (BX + 1) + tx + 1] - fa[ty * (BX + 1) + tx]) +
                 (fa[S::PFX + (ty + 1) * BX + tx] - fa[S::PFX + ty * BX + tx]);
        const Real* sp = s_phi + a * C2;
        gc[a][0] = Real(0.5) * (sp[r2 + 1] - sp[r2 - 1]);
        gc[a][1] = Real(0.5) * (sp[r2 + W2] - sp[r2 - W2]);
      }
      Real dadphi[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) dadphi[a] = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a)
#pragma unroll
        for (int b = a + 1; b < NP; ++b) {
          // a phase absent from the 3x3 neighbourhood: q = 0, exactly 0
          const Real gab = P.gamma[a][b];
          if (gab == Real(0) || (act & ((1u << a) | (1u << b))) != ((1u << a) | (1u << b))) continue;
          Real q[2], v[2];
          q[0] = ph[a] * gc[b][0] - ph[b] * gc[a][0];
          q[1] = ph[a] * gc[b][1] - ph[b] * gc[a][1];
          dAdq_vec_pair<2, EXT>(P, a, b, q, v);
          dadphi[a] += gab * (v[0] * gc[b][0] + v[1] * gc[b][1]);
          dadphi[b] -= gab * (v[0] * gc[a][0] + v[1] * gc[a][1]);
        }
      const Real theta = theta_base + P.G * Real(fy);
      Real psi[NP];
#pragma unroll
      for (int b = 0; b < NP; ++b) {
        Real sv = P.S[b] * theta;
#pragma unroll
        for (int i = 0; i < NC; ++i) sv -= mu[i] * mu[i] * P.inv4A[b] + mu[i] * ceq_of(b, i, fy);
        psi[b] = sv;
      }
      Real rate[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        Real obst = Real(0), drv = Real(0);
#pragma unroll
        for (int b = 0; b < NP; ++b) {
          if (b != a) obst += P.gamma[a][b] * ph[b];
          drv += psi[b] * interp_dh<NP>(ph, b, a);
        }
        rate[a] = P.eps * (div[a] - dadphi[a]) - P.obst * obst - drv;
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
      Real uv[NP];
      int m = 0;
#pragma unroll
      for (int a = 0; a < NP; ++a)
        if (act & (1u << a)) uv[m++] = ph[a] + P.mob_eps * (rate[a] - lam);
      if (NP == 2) {
        Real sv = uv[1];
        sv = sv < Real(0) ? Real(0) : (sv > Real(1) ? Real(1) : sv);
        out[1] = sv;
        out[0] = Real(1) - sv;
      } else {
        project_simplex<Real, NP>(uv, m);
        m = 0;
#pragma unroll
        for (int a = 0; a < NP; ++a) out[a] = (act & (1u << a)) ? uv[m++] : Real(0);
      }
    }
  }
  bool changed = false;
  int pure = -1;  // the phase at exactly 1 when every other phase is exactly 0
  {
    int n1 = 0, n0 = 0;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      s_pn[a * NT + tid] = out[a];
      changed = changed || out[a] != ph[a];
      if (out[a] == Real(1)) {
        pure = a;
        ++n1;
      } else if (out[a] == Real(0)) {
        ++n0;
      }
    }
    if (n1 != 1 || n0 != NP - 1) pure = -1;
  }
  s_chg[tid] = changed ? 1 : 0;
  // h of a pure cell is the unit vector of its phase, exactly
  s_hl[tid] = pure >= 0 ? (pure == 0 ? Real(1) : Real(0)) : interp_h<NP>(out, 0);
  if constexpr (SHRINK) {
    // F_S = sum_a eta_a (phi_a^{n+1} - phi_a^n) grad phi_a^n / |grad phi_a^n|
    Real fsx = Real(0), fsy = Real(0);
    if (changed) {
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        if (P.eta[a] == Real(0)) continue;
        const Real* sp = s_phi + a * C2;
        const Real gxa = Real(0.5) * (sp[r2 + 1] - sp[r2 - 1]);
        const Real gya = Real(0.5) * (sp[r2 + W2] - sp[r2 - W2]);
        const Real g2 = gxa * gxa + gya * gya;
        if (g2 <= Real(1e-12)) continue;
        const Real ig = Real(1) / sqrt(g2);
        const Real rate = out[a] - ph[a];
        fsx += P.eta[a] * rate * gxa * ig;
        fsy += P.eta[a] * rate * gya * ig;
      }
    }
    Real dk[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) dk[k] = Codec<Store>::load(s_fs[k * NT + tid]);
    lbm_cell(dk, fsx, fsy);
  }
  const bool any_changed = __syncthreads_or(changed);

  // 2. solute flux through the +x face (slot tid) and the +y face (slot NT +
  //    tid): -M_f (mu_b - mu_a) - a eps sum_{a>0} [phi_l]_f [c_l - c_a]_f
  //    [dphi_a]_f n_a.e_d + [U_d h_l c_l]_f; zero through walls, obstacle
  //    cells and past a ragged edge
  auto mu_face = [&](int d) {
    const int nb = d == 0 ? tid + 1 : tid + BX;  // neighbour thread
    const int nr = d == 0 ? r2 + 1 : r2 + W2;    // neighbour in R1-plus-ring
    const int gbd = (d == 0 ? gx : gy) + 1;      // global index of the upper cell
    bool closed = (P.bc[d] == kWall && (gbd == 0 || gbd == P.n[d])) || gbd > P.n[d];
    if (!closed && (P.wall[0] | P.wall[1])) {
      const int ux_ = d == 0 ? fold_axis(P, gx + 1, 0) : fx;
      const int uy_ = d == 0 ? fy : fold_axis(P, gy + 1, 1);
      closed = obs || obstacle(P, ux_, uy_, 0);
    }
    Real J[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) J[i] = Real(0);
    if (!closed) {
      const Real Mf = Real(0.5) * P.M0 * (s_pn[tid] + s_pn[nb]);  // plane 0 = liquid
      const Real ua = s_u[d * NT + tid] * s_hl[tid], ub = s_u[d * NT + nb] * s_hl[nb];
      // vertical index of the neighbour (for ceq(T))
      const int vb = d == 0 ? fy : (inner_tile ? fy + 1 : fold_axis(P, gy + 1, 1));
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        const Real ma = s_mu[i * NT + tid], mb = s_mu[i * NT + nb];
        J[i] = -Mf * (mb - ma) + Real(0.5) * (ua * (ceq_of(0, i, fy) + ma * P.inv2A[0]) +
                                              ub * (ceq_of(0, i, vb) + mb * P.inv2A[0]));
      }
      // the current carries phi_l's face value as a factor of every term: on a
      // face without liquid it is exactly 0 and skipped
      const Real liq = any_changed && P.at_eps != Real(0) && (s_chg[tid] | s_chg[nb])
                           ? Real(0.5) * (s_phi[r2] + s_phi[nr])
                           : Real(0);
      if (liq != Real(0)) {
        const int st = d == 0 ? W2 : 1;  // transverse stride
        Real at[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) at[i] = Real(0);
#pragma unroll
        for (int a = 1; a < NP; ++a) {
          const Real* sp = s_phi + a * C2;
          const Real gn = sp[nr] - sp[r2];
          const Real gt = Real(0.25) * (sp[r2 + st] + sp[nr + st] - sp[r2 - st] - sp[nr - st]);
          const Real g2 = gn * gn + gt * gt;
          if (g2 <= Real(1e-12)) continue;
          const Real nd = liq * gn / sqrt(g2);
          const Real dphi = Real(0.5) * ((s_pn[a * NT + tid] - sp[r2]) + (s_pn[a * NT + nb] - sp[nr]));
          const Real dinv = P.inv2A[0] - P.inv2A[a];
#pragma unroll
          for (int i = 0; i < NC; ++i) {
            Real dc = (P.ceq[0][i] - P.ceq[a][i]) +
                      Real(0.5) * (s_mu[i * NT + tid] + s_mu[i * NT + nb]) * dinv;
            if constexpr (EXT) {
              const int vb = d == 0 ? fy : (inner_tile ? fy + 1 : fold_axis(P, gy + 1, 1));
              dc += (P.dceq_dT[0][i] - P.dceq_dT[a][i]) *
                    (theta_base + Real(0.5) * P.G * Real(fy + vb));
            }
            at[i] += dc * dphi * nd;
          }
        }
#pragma unroll
        for (int i = 0; i < NC; ++i) J[i] -= P.at_eps * at[i];
      }
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) s_flux[i * 2 * NT + d * NT + tid] = J[i];
  };
  if (tx < BX - 1) mu_face(0);
  if (ty < BY - 1) mu_face(1);
  __syncthreads();

  // 3. inner cells: mu^{n+1}, phi^{n+1}, pulled f^{n+1}
  if (!inner) return;
#pragma unroll
  for (int sidx = 0; sidx < NS; ++sidx) (phi_out + sidx * P.plane)[g] = out[NP == 2 ? 1 : sidx];
  if (obs) {
#pragma unroll
    for (int i = 0; i < NC; ++i) (mu_out + i * P.plane)[g] = mu[i];
  } else if (!EXT && !changed && pure >= 0) {
    // unchanged pure cell: source term exactly 0, chi = 1 / (2 A_pure)
    Real ichi = P.chi_pure[0];
#pragma unroll
    for (int a = 1; a < NP; ++a)
      if (pure == a) ichi = P.chi_pure[a];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const Real* Ji = s_flux + i * 2 * NT;
      const Real div = (Ji[tid] - Ji[tid - 1]) + (Ji[NT + tid] - Ji[NT + tid - BX]);
      (mu_out + i * P.plane)[g] = mu[i] + (-div - Real(0)) * ichi;
    }
  } else {
    Real chi = Real(0), hn[NP], ho[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      hn[a] = interp_h<NP>(out, a);
      ho[a] = changed ? interp_h<NP>(ph, a) : hn[a];
      chi += hn[a] * P.inv2A[a];
    }
    const Real ichi = rcp_rn(chi);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const Real* Ji = s_flux + i * 2 * NT;
      const Real div = (Ji[tid] - Ji[tid - 1]) + (Ji[NT + tid] - Ji[NT + tid - BX]);
      Real src = Real(0);
      if (changed) {
#pragma unroll
        for (int a = 0; a < NP; ++a) src += (ceq_of(a, i, fy) + mu[i] * P.inv2A[a]) * (hn[a] - ho[a]);
      }
      if constexpr (EXT) {
        // -(dT/dt) sum_a (dc_a/dT)_mu h_a^{n+1}, dT/dt = -G V
#pragma unroll
        for (int a = 0; a < NP; ++a) src -= Real(P.GV) * P.dceq_dT[a][i] * hn[a];
      }
      (mu_out + i * P.plane)[g] = mu[i] + (-div - src) * ichi;
    }
  }
  pull_f();
}

}  // namespace gpflbm

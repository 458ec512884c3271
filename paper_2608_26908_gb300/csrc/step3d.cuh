// Fused 3D step for sm_103a, the general path (Algorithm 1: phase field,
// chemical potential, lattice Boltzmann).  Tiles whose reach is pure liquid
// take the lean path of step3d_liquid.cuh instead; the kernels that run the
// two are at the end of that file.
//
// A CTA owns an xy tile and a z segment of ZS planes.  It runs one thread per
// cell of the tile's one-cell xy halo region ("R1", BX x BY columns) and
// marches up the segment plane by plane, keeping the planes each stage
// still needs in shared-memory rings.  At lead plane L it
//   A. reads phi^n of plane L (its column and, for the first threads, the
//      ring of columns around R1) and records which phases are present;
//   B. reads mu^n and f^n of plane C = L-1, forms rho, the implicit-drag
//      velocity U and the forces, and, for the tile's inner columns of the
//      owned planes, collides the populations (BGK + Guo) and pushes them to
//      x + c_k of f^{n+1} in global memory (halfway bounce-back at walls);
//   C. updates the phase field of plane C where phases mix (face fluxes,
//      Lambda over the present phases, Gibbs-simplex projection);
//   D. forms the solute fluxes of plane M = L-2 (in-plane faces and the face
//      to plane M+1; the face to M-1 comes from the previous plane) and
//      writes mu^{n+1}, phi^{n+1} of plane M.
// Pushing instead of pulling means each cell is collided once, by the CTA
// that owns it, and no collided populations are staged.
#pragma once

#include "gpflbm_kernels.cuh"

namespace gpflbm {

// Tiles of the 3D step: BX x BY threads (BX-2 x BY-2 owned columns), ZS
// planes a CTA.  FP32: six planes, measured best on both 3D workloads
// (ternary eutectic 1.82 ms a step against 1.89 / 1.98 ms at 8 / 16 planes;
// dendrite 0.670 ms against 0.689 / 0.715), although a CTA's march then
// repeats a larger share of halo planes: the marches are short, the grid
// is deep, and no general tile, whose lone march sets the step's tail,
// runs long.
template <class Real>
struct Block3D;
template <>
struct Block3D<float> {
  static constexpr int BX = 32, BY = 16, ZS = 6;
};
template <>
struct Block3D<double> {
  static constexpr int BX = 32, BY = 8, ZS = 16;
};

template <int NP, int NC, class Real, class Store, int QQ = 19>
struct Step3D {
  static constexpr int BX = Block3D<Real>::BX, BY = Block3D<Real>::BY, ZS = Block3D<Real>::ZS;
  static constexpr int NT = BX * BY, Q = QQ;  // D3Q19 or D3Q27
  static constexpr int NS = PhiStore<NP>::NS;
  // resident CTAs per SM the register budget is cut for: two (64 registers)
  // on D3Q19 in FP32, for any number of phases (three and four phases spill
  // a few dozen bytes, yet two CTAs of 64 registers beat one of 128: 1.79
  // against 1.91 ms on the ternary eutectic); FP64 and 27 populations: one
  static constexpr int MIN_CTAS = (sizeof(Real) == 4 && QQ == 19) ? 2 : 1;
  // both paths in one launch where they have the same register budget and
  // the general path's shared memory is small (two phases: 46 KB).  A launch
  // reserves its largest path's shared memory for every CTA, and with more
  // phases (96 KB) the liquid tiles are left too little L1 for their loads
  // in flight: the ternary eutectic takes 1.88 ms a step in one launch,
  // 1.77 ms in two.
  static constexpr bool ONE_LAUNCH = MIN_CTAS == 2 && NP == 2;
  static constexpr int OX = BX - 2, OY = BY - 2;
  static constexpr int W2 = BX + 2, H2 = BY + 2, C2 = W2 * H2;
  static constexpr int RING = C2 - NT;
  static constexpr int PFX = (BX + 1) * BY, PFY = BX * (BY + 1);  // in-plane phase-field faces
  static constexpr size_t al(size_t v) { return (v + 15) / 16 * 16; }
  static constexpr size_t phi = 0;                                  // 4 planes x NS x C2
  static constexpr size_t mask = al(phi + sizeof(Real) * 4 * NS * C2);  // 3 planes x C2
  // phi^{n+1} of planes C and M (written in C, read by the solute faces
  // and the update of the next iteration); U_x, U_y of the same two planes
  // (U_z only enters this column's own z-face: registers)
  static constexpr size_t pn = al(mask + 3 * C2);                   // 2 planes x NP x NT
  static constexpr size_t u = al(pn + sizeof(Real) * 2 * NP * NT);   // 2 planes x 2 x NT
  static constexpr size_t mu = al(u + sizeof(Real) * 2 * 2 * NT);    // 2 planes x NC x NT
  static constexpr size_t hl = al(mu + sizeof(Real) * 2 * NC * NT);  // 2 planes x NT
  static constexpr size_t chg = al(hl + sizeof(Real) * 2 * NT);      // 2 planes x NT bytes
  static constexpr size_t flux = al(chg + 2 * NT);                   // PF or solute in-plane faces
  static constexpr size_t flux_n =
      NP * (PFX + PFY) > 2 * NC * NT ? NP * (PFX + PFY) : 2 * NC * NT;
  static constexpr size_t bytes = al(flux + sizeof(Real) * flux_n);
};

struct Step3DIO {
  const void* phi_in;
  void* phi_out;
  const void* mu_in;
  void* mu_out;
  const void* f_in;
  void* f_out;
  const double* clock_in;
  double* clock_out;
  const unsigned char* flags_in;  // liquid flag per tile of the input state
  unsigned char* flags_out;       // ... of the output state
};

// EXT: the extended model -- pairs' crystal axes turned about z (dAdq_pair)
// and equilibrium compositions ceq_a(T) with the temperature term of Eq. conc.
// SHRINK: the shrinkage force needs phi^{n+1}, so the collision of a plane
// moves after its phase-field update (its populations are read again then).
// The general path for one tile: xy tile (bx, by) of a gxt x gyt tiling,
// z segment bz.  The kernels that run it are at the end of step3d_liquid.cuh.
template <int NP, int NC, class Real, class Store, bool SHRINK, int QQ, bool EXT>
__device__ __forceinline__ void general_tile(const DevParams<Real>& P, const Step3DIO& io, int bx, int by, int bz,
                                             int gxt, int gyt) {
  using S = Step3D<NP, NC, Real, Store, QQ>;
  using Lat = Lattice<QQ>;
  constexpr int BX = S::BX, BY = S::BY, ZS = S::ZS, NT = S::NT, Q = QQ;
  constexpr int W2 = S::W2, H2 = S::H2, C2 = S::C2, NS = S::NS;
  extern __shared__ __align__(16) unsigned char smem[];
  Real* s_phi = reinterpret_cast<Real*>(smem + S::phi);
  unsigned char* s_mask = smem + S::mask;
  Real* s_pn = reinterpret_cast<Real*>(smem + S::pn);
  Real* s_u = reinterpret_cast<Real*>(smem + S::u);
  Real* s_mu = reinterpret_cast<Real*>(smem + S::mu);
  Real* s_hl = reinterpret_cast<Real*>(smem + S::hl);
  unsigned char* s_chg = smem + S::chg;
  Real* s_flux = reinterpret_cast<Real*>(smem + S::flux);

  const Real* __restrict__ phi_in = static_cast<const Real*>(io.phi_in);
  const Real* __restrict__ mu_in = static_cast<const Real*>(io.mu_in);
  const Store* __restrict__ f_in = static_cast<const Store*>(io.f_in);
  Real* __restrict__ phi_out = static_cast<Real*>(io.phi_out);
  Real* __restrict__ mu_out = static_cast<Real*>(io.mu_out);
  Store* __restrict__ f_out = static_cast<Store*>(io.f_out);

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2], px = P.px;
  const int zst = px * ny;  // plane stride (a plane holds fewer than 2^31 cells)
  // z segments start at the first owned plane (v_lo = 0 for a whole grid;
  // a slab owns planes v_lo .. v_hi - 1 of the vertical axis)
  const int x0 = bx * S::OX, y0 = by * S::OY, z0 = P.v_lo + bz * ZS;
  const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
  const bool inner_xy = x0 >= 2 && x0 - 2 + W2 <= nx && y0 >= 2 && y0 - 2 + H2 <= ny;
  const int fx = inner_xy ? gx : fold_axis(P, gx, 0);
  const int fy = inner_xy ? gy : fold_axis(P, gy, 1);
  const int gxy = fy * px + fx;
  const int r2 = (ty + 1) * W2 + tx + 1;
  // inner columns of the tile write the tile's cells
  const bool owner = tx >= 1 && tx <= BX - 2 && ty >= 1 && ty <= BY - 2 && gx < nx && gy < ny;
  const double t_now = io.clock_in[0];
  if (bx == 0 && by == 0 && bz == 0 && tid == 0) io.clock_out[0] = t_now + 1.0;
  const Real theta_base = Real(P.theta0) - Real(P.GV) * Real(t_now);
  // EXT: ceq_a,i(T) at vertical index v, T - T_E = theta_base + G v
  auto ceq_of = [&](int a, int i, int v) -> Real {
    if constexpr (EXT)
      return fma_rn(P.dceq_dT[a][i], fma_rn(P.G, Real(v), theta_base), P.ceq[a][i]);
    else
      return P.ceq[a][i];
  };
  const bool has_walls = (P.wall[0] | P.wall[1] | P.wall[2]) != 0;  // obstacle rows
  // vertical index of a plane the kernel reads: folded on the whole grid
  // (walls mirror, periodic wraps), then kept inside the planes the buffers
  // hold (v_lo - 2 .. v_hi + 1; for a whole grid the fold already is); the
  // buffers start at plane zbase (0, or v_lo - 2 for a slab with halos)
  auto vz = [&](int v) {
    const int f = fold_axis(P, v, 2);
    return f < P.v_lo - 2 ? P.v_lo - 2 : (f > P.v_hi + 1 ? P.v_hi + 1 : f);
  };
  auto zrow = [&](int fz) { return (fz - P.zbase) * zst; };

  int rx = 0, ry = 0;  // ring column held by threads tid < RING
  int gring = 0;
  if (tid < S::RING) {
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
    const int qx = inner_xy ? x0 - 2 + rx : fold_axis(P, x0 - 2 + rx, 0);
    const int qy = inner_xy ? y0 - 2 + ry : fold_axis(P, y0 - 2 + ry, 1);
    gring = qy * px + qx;
  }
  const int rr2 = ry * W2 + rx;

  auto slot4 = [](int p) { return p & 3; };
  // (p + 3) mod 3; v / 3 = umulhi(v, 0xAAAAAAAB) >> 1 for every 32-bit v
  auto slot3 = [](int p) {
    const unsigned v = (unsigned)(p + 3);
    return (int)(v - 3u * (__umulhi(v, 0xAAAAAAABu) >> 1));
  };
  auto slot2 = [](int p) { return p & 1; };
  // phase a of plane p (ring of four) at R1-plus-ring index i
  auto PH = [&](int p, int a, int i) -> Real {
    const Real* b = s_phi + slot4(p) * NS * C2;
    if (NP == 2) return a == 0 ? Real(1) - b[i] : b[i];
    return b[a * C2 + i];
  };
  auto MK = [&](int p, int i) -> unsigned { return s_mask[slot3(p) * C2 + i]; };
  // a cell of pure liquid: phi_0 = 1 and every other phase 0, exactly
  auto pure_liquid = [](const Real* v) {
    bool p = v[0] == Real(1);
#pragma unroll
    for (int a = 1; a < NP; ++a) p = p && v[a] == Real(0);
    return p;
  };
  // Liquid planes: bit 0 = plane L, bit 1 = C, bit 2 = M, bit 3 = M - 1 is
  // set when every cell of that plane in R1 and its ring is pure liquid and
  // no cell of R1 is an obstacle (the whole CTA agrees: __syncthreads_and).
  // The shrinkage variant keeps the general path everywhere (its registers
  // are already spent on the deferred collision).
  constexpr bool LIQ = !SHRINK;
  unsigned liq_hist = 0;

  // every phase value this thread writes in the plane is pure liquid (for
  // the tile's flag of that plane)
  bool out_liq = true;

  // OR of the phase masks over the 3x3 in-plane neighbourhood of this
  // column, for planes C-1 and C (carried) and L (new)
  unsigned xy_m1 = 0, xy_0 = 0;

  // phase-field z-face fluxes of this column: (C-1, C) carried, (C, C+1) new
  Real pfz_lo[NP], pfz_hi[NP];
  // solute z-face fluxes of this column: (M-1, M) carried, (M, M+1) new
  Real mz_lo[NC], mz_hi[NC];
  // U_z of this column in planes M and C
  Real uz_M = Real(0), uz_C = Real(0);
#pragma unroll
  for (int a = 0; a < NP; ++a) pfz_lo[a] = pfz_hi[a] = Real(0);
#pragma unroll
  for (int i = 0; i < NC; ++i) mz_lo[i] = mz_hi[i] = Real(0);

  // face flux of the phase field between cells A and B (R1-plus-ring indices
  // in planes pa, pb); normal axis d; t1, t2 the transverse steps (in-plane
  // index offsets or plane offsets); returns the d-th component of
  // -sum_{b != a} gamma_ab phi_b dA/dq(q_ab) for every phase
  auto pf_flux = [&](int pa, int ia, int pb, int ib, int d, bool closed, Real* fl) {
#pragma unroll
    for (int a = 0; a < NP; ++a) fl[a] = Real(0);
    // the cells the stencil reads
    unsigned grp;
    Real pf[NP], g3[NP][3];
    if (d == 2) {
      grp = MK(pa, ia) | MK(pb, ib) | MK(pa, ia + 1) | MK(pb, ib + 1) | MK(pa, ia - 1) |
            MK(pb, ib - 1) | MK(pa, ia + W2) | MK(pb, ib + W2) | MK(pa, ia - W2) | MK(pb, ib - W2);
    } else {
      const int st = d == 0 ? W2 : 1;
      grp = MK(pa, ia) | MK(pb, ib) | MK(pa, ia + st) | MK(pb, ib + st) | MK(pa, ia - st) |
            MK(pb, ib - st) | MK(pa - 1, ia) | MK(pb - 1, ib) | MK(pa + 1, ia) | MK(pb + 1, ib);
    }
    if (__popc(grp) < 2 || closed) return;
    // A phase whose mask bit is clear in every cell the stencil reads is
    // exactly 0 there: its face value and gradient are 0, so every pair it
    // belongs to has q = 0 and contributes exactly 0.  Such phases and pairs
    // are skipped (two or three of the four phases at most interfaces).
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      pf[a] = Real(0);
      g3[a][0] = g3[a][1] = g3[a][2] = Real(0);
      if (!(grp & (1u << a))) continue;
      const Real va = PH(pa, a, ia), vb = PH(pb, a, ib);
      pf[a] = Real(0.5) * (va + vb);
      g3[a][d] = vb - va;
      if (!P.aniso) continue;  // dA/dq = 2 q: only q_d enters the flux
      if (d == 2) {
        g3[a][0] = Real(0.25) * (PH(pa, a, ia + 1) + PH(pb, a, ib + 1) - PH(pa, a, ia - 1) - PH(pb, a, ib - 1));
        g3[a][1] = Real(0.25) * (PH(pa, a, ia + W2) + PH(pb, a, ib + W2) - PH(pa, a, ia - W2) - PH(pb, a, ib - W2));
      } else {
        const int st = d == 0 ? W2 : 1;  // the other in-plane axis
        g3[a][1 - d] = Real(0.25) * (PH(pa, a, ia + st) + PH(pb, a, ib + st) - PH(pa, a, ia - st) - PH(pb, a, ib - st));
        g3[a][2] = Real(0.25) * (PH(pa + 1, a, ia) + PH(pb + 1, a, ib) - PH(pa - 1, a, ia) - PH(pb - 1, a, ib));
      }
    }
#pragma unroll
    for (int a = 0; a < NP; ++a)
#pragma unroll
      for (int b = a + 1; b < NP; ++b) {
        const Real gab = P.gamma[a][b];
        if (gab == Real(0) || (grp & ((1u << a) | (1u << b))) != ((1u << a) | (1u << b))) continue;
        Real q[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) q[t] = pf[a] * g3[b][t] - pf[b] * g3[a][t];
        const Real v = dAdq_pair<3, EXT>(P, a, b, q, d);
        fl[a] -= gab * pf[b] * v;
        fl[b] += gab * pf[a] * v;
      }
  };

  const int L0 = z0 - 2, L1 = z0 + ZS + 1;
  for (int L = L0; L <= L1; ++L) {
    const int C = L - 1, M = L - 2;
    uz_M = uz_C;  // plane C of the previous iteration is this one's M
    bool liq_l;  // this thread's cells of plane L are pure liquid
    // A. phi^n of plane L
    {
      const int zo = zrow(vz(L));
      Real* b = s_phi + slot4(L) * NS * C2;
      unsigned m = 0;
      Real v[NP];
      load_phases<NP>(phi_in, zo + gxy, P.plane, v);
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        if (NP != 2 || a == 1) b[(NP == 2 ? 0 : a) * C2 + r2] = v[a];
        if (v[a] > Real(0)) m |= 1u << a;
      }
      s_mask[slot3(L) * C2 + r2] = (unsigned char)m;
      liq_l = pure_liquid(v) && !(has_walls && obstacle(P, fx, fy, vz(L)));
      if (tid < S::RING) {
        load_phases<NP>(phi_in, zo + gring, P.plane, v);
        liq_l = liq_l && pure_liquid(v);
        m = 0;
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          if (NP != 2 || a == 1) b[(NP == 2 ? 0 : a) * C2 + rr2] = v[a];
          if (v[a] > Real(0)) m |= 1u << a;
        }
        s_mask[slot3(L) * C2 + rr2] = (unsigned char)m;
      }
    }
    // B. moments, U and (owned planes, inner columns) collision + push, plane C
    const bool doC = C >= z0 - 1 && C <= z0 + ZS;
    if (doC) {
      const int fzc = vz(C);
      const int gi = zrow(fzc) + gxy;  // the buffers hold fewer than 2^31 cells a plane
      const bool obs = has_walls && obstacle(P, fx, fy, fzc);
      Real mu[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        mu[i] = (mu_in + i * P.plane)[gi];
        s_mu[(slot2(C) * NC + i) * NT + tid] = mu[i];
      }
      if constexpr (!SHRINK) {
      Real dk[Q];
#pragma unroll
      for (int k = 0; k < Q; ++k) dk[k] = Codec<Store>::load(at_bytes(f_in + gi, P.f_at[k]));
      Real drho = Real(0), m3[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        drho += dk[k];
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (Lat::c(k, a) != 0) m3[a] += Real(Lat::c(k, a)) * dk[k];
      }
      const Real rho = Real(1) + drho;
      // phi_l^n of this cell (plane C was read as plane L one step earlier)
      const Real phl = obs ? Real(0) : PH(C, 0, r2);
      const Real drive = buoyancy_drive<NC, EXT>(P, fma_rn(P.G, Real(fzc), theta_base), mu);
      Real u[3], F[3];
      force_velocity<3>(P, rho, phl, drive, m3, u, F);
#pragma unroll
      for (int a = 0; a < 2; ++a) s_u[(slot2(C) * 2 + a) * NT + tid] = u[a];
      uz_C = u[2];
      // A slab also collides the cells of its halo planes next to a
      // neighbouring slab and keeps only the populations that stream into
      // its own planes (hdir = +1 below, -1 above): the same values the
      // neighbour computes for those cells, so nothing crosses after the step.
      int hdir = 0;
      if (C == P.v_lo - 1 && P.v_lo > 0 && C == z0 - 1) hdir = 1;
      if (C == P.v_hi && P.v_hi < nz && C - 1 >= z0 && C - 1 < z0 + ZS) hdir = -1;
      if (owner && ((C >= z0 && C < z0 + ZS && C < P.v_hi) || hdir != 0)) {
        const bool inner_z = C >= 1 && C + 1 < nz;
        if (inner_xy && inner_z) {
          // x + c_k is inside the grid: population k lands at gi + c_k . (1, px, zst)
          Store* const fo = f_out + gi;
          collide<Q>(P, dk, drho, rho, u, F, [&](int k, Real val) {
            if (hdir != 0 && Lat::c(k, 2) != hdir) return;
            at_bytes(fo, P.f_to[k]) = Codec<Store>::put(val);
          });
        } else {
        // push to x + c_k (periodic axes wrap; across a wall the population
        // returns reversed into the cell)
        const PushAxis X = push_axis(gx, nx, P.bc[0] == kWall, 1);
        const PushAxis Y = push_axis(gy, ny, P.bc[1] == kWall, px);
        const PushAxis Z = push_axis(C, nz, P.bc[2] == kWall, zst);
        collide<Q>(P, dk, drho, rho, u, F, [&](int k, Real val) {
          if (hdir != 0 && Lat::c(k, 2) != hdir) return;
          push_store<Lat>(f_out, P.plane, gi, k, Codec<Store>::put(val), X, Y, Z);
        });
        }
      }
      }  // !SHRINK
    }
    if constexpr (LIQ)
      liq_hist = ((liq_hist << 1) | (__syncthreads_and(liq_l) ? 1u : 0u)) & 15u;
    else
      __syncthreads();

    // C. phase field of plane C where phases mix
    const bool pfC = C >= z0 - 1 && C <= z0 + ZS;
    Real out[NP];
    bool mixed = false, multi = false;
    unsigned act = 0;
    unsigned xy_l = 0;
    if (liq_hist & 1u) {
      xy_l = 1u;  // plane L is liquid: every mask of the 3x3 is the liquid bit
    } else {
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) xy_l |= MK(L, r2 + dy * W2 + dx);
    }
    act = xy_m1 | xy_0 | xy_l;  // the 3x3x3 neighbourhood of plane C
    xy_m1 = xy_0;
    xy_0 = xy_l;
    if (pfC) {
      const int fzc = vz(C);
      mixed = __popc(act) >= 2;
      multi = mixed && !(has_walls && obstacle(P, fx, fy, fzc));
#pragma unroll
      for (int a = 0; a < NP; ++a) out[a] = PH(C, a, r2);
    }
    // A face flux reads cells inside the 3x3x3 neighbourhood of its cell in
    // plane C, so with no mixed neighbourhood in the plane every face of the
    // plane (and the z-face above it) is exactly zero.
    // (planes C-1, C and L all liquid: nothing mixes, and the CTA knows it
    // without another barrier)
    if ((liq_hist & 7u) == 7u || !__syncthreads_or(pfC && mixed)) {
#pragma unroll
      for (int a = 0; a < NP; ++a) pfz_hi[a] = Real(0);
    } else {
      if (pfC) {
        // in-plane faces of plane C into shared memory
        Real fl[NP];
        const bool cx_hi = P.bc[0] == kWall && (gx + 1 == 0 || gx + 1 == nx);
        pf_flux(C, r2, C, r2 + 1, 0, cx_hi, fl);
#pragma unroll
        for (int a = 0; a < NP; ++a) s_flux[a * (S::PFX + S::PFY) + ty * (BX + 1) + tx + 1] = fl[a];
        if (tx == 0) {
          const bool cx_lo = P.bc[0] == kWall && (gx == 0 || gx == nx);
          pf_flux(C, r2 - 1, C, r2, 0, cx_lo, fl);
#pragma unroll
          for (int a = 0; a < NP; ++a) s_flux[a * (S::PFX + S::PFY) + ty * (BX + 1)] = fl[a];
        }
        const bool cy_hi = P.bc[1] == kWall && (gy + 1 == 0 || gy + 1 == ny);
        pf_flux(C, r2, C, r2 + W2, 1, cy_hi, fl);
#pragma unroll
        for (int a = 0; a < NP; ++a) s_flux[a * (S::PFX + S::PFY) + S::PFX + (ty + 1) * BX + tx] = fl[a];
        if (ty == 0) {
          const bool cy_lo = P.bc[1] == kWall && (gy == 0 || gy == ny);
          pf_flux(C, r2 - W2, C, r2, 1, cy_lo, fl);
#pragma unroll
          for (int a = 0; a < NP; ++a) s_flux[a * (S::PFX + S::PFY) + S::PFX + tx] = fl[a];
        }
        // z-faces of this column: (C, C+1), and (C-1, C) on the first plane
        const bool cz_hi = P.bc[2] == kWall && (C + 1 == 0 || C + 1 == nz);
        pf_flux(C, r2, C + 1, r2, 2, cz_hi, pfz_hi);
        if (C == z0 - 1) {
          const bool cz_lo = P.bc[2] == kWall && (C == 0 || C == nz);
          pf_flux(C - 1, r2, C, r2, 2, cz_lo, pfz_lo);
        }
      }
      __syncthreads();
      if (pfC && multi) {
        Real div[NP], gc[NP][3];
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          const Real* fa = s_flux + a * (S::PFX + S::PFY);
          div[a] = (fa[ty * (BX + 1) + tx + 1] - fa[ty * (BX + 1) + tx]) +
                   (fa[S::PFX + (ty + 1) * BX + tx] - fa[S::PFX + ty * BX + tx]) + (pfz_hi[a] - pfz_lo[a]);
          // a phase absent from the 3x3x3 neighbourhood has a zero central
          // gradient, and its pairs contribute exactly 0 below
          gc[a][0] = gc[a][1] = gc[a][2] = Real(0);
          if (!(act & (1u << a))) continue;
          gc[a][0] = Real(0.5) * (PH(C, a, r2 + 1) - PH(C, a, r2 - 1));
          gc[a][1] = Real(0.5) * (PH(C, a, r2 + W2) - PH(C, a, r2 - W2));
          gc[a][2] = Real(0.5) * (PH(C + 1, a, r2) - PH(C - 1, a, r2));
        }
        Real ph[NP];
#pragma unroll
        for (int a = 0; a < NP; ++a) ph[a] = out[a];
        Real dadphi[NP];
#pragma unroll
        for (int a = 0; a < NP; ++a) dadphi[a] = Real(0);
#pragma unroll
        for (int a = 0; a < NP; ++a)
#pragma unroll
          for (int b = a + 1; b < NP; ++b) {
            const Real gab = P.gamma[a][b];
            if (gab == Real(0) || (act & ((1u << a) | (1u << b))) != ((1u << a) | (1u << b))) continue;
            Real q[3], v[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) q[t] = ph[a] * gc[b][t] - ph[b] * gc[a][t];
            dAdq_vec_pair<3, EXT>(P, a, b, q, v);
            dadphi[a] += gab * (v[0] * gc[b][0] + v[1] * gc[b][1] + v[2] * gc[b][2]);
            dadphi[b] -= gab * (v[0] * gc[a][0] + v[1] * gc[a][1] + v[2] * gc[a][2]);
          }
        const int fzC = vz(C);
        const Real theta = theta_base + P.G * Real(fzC);
        Real mu[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) mu[i] = s_mu[(slot2(C) * NC + i) * NT + tid];
        Real psi[NP];
#pragma unroll
        for (int b = 0; b < NP; ++b) {
          Real sv = P.S[b] * theta;
#pragma unroll
          for (int i = 0; i < NC; ++i) sv -= mu[i] * mu[i] * P.inv4A[b] + mu[i] * ceq_of(b, i, fzC);
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
    if (pfC) {
      bool changed = false;
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        s_pn[(slot2(C) * NP + a) * NT + tid] = out[a];
        changed = changed || out[a] != PH(C, a, r2);
      }
      if constexpr (SHRINK) {
        // F_S = sum_a eta_a (phi_a^{n+1} - phi_a^n) grad phi_a^n / |grad phi_a^n|
        Real fs[3] = {Real(0), Real(0), Real(0)};
        if (changed) {
#pragma unroll
          for (int a = 0; a < NP; ++a) {
            if (P.eta[a] == Real(0)) continue;
            Real gr[3];
            gr[0] = Real(0.5) * (PH(C, a, r2 + 1) - PH(C, a, r2 - 1));
            gr[1] = Real(0.5) * (PH(C, a, r2 + W2) - PH(C, a, r2 - W2));
            gr[2] = Real(0.5) * (PH(C + 1, a, r2) - PH(C - 1, a, r2));
            const Real g2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
            if (g2 <= Real(1e-12)) continue;
            const Real ig = Real(1) / sqrt(g2);
            const Real rate = out[a] - PH(C, a, r2);
#pragma unroll
            for (int t = 0; t < 3; ++t) fs[t] += P.eta[a] * rate * gr[t] * ig;
          }
        }
        // moments, U and F with the shrinkage force, collision + push (as phase B)
        const int fzc = vz(C);
        const int gi = zrow(fzc) + gxy;
        const bool obs = has_walls && obstacle(P, fx, fy, fzc);
        Real dk[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) dk[k] = Codec<Store>::load(at_bytes(f_in + gi, P.f_at[k]));
        Real drho = Real(0), m3[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          drho += dk[k];
#pragma unroll
          for (int a = 0; a < 3; ++a)
            if (Lat::c(k, a) != 0) m3[a] += Real(Lat::c(k, a)) * dk[k];
        }
        const Real rho = Real(1) + drho;
        const Real phl = obs ? Real(0) : PH(C, 0, r2);
        const Real sl = Real(1) - phl;
        const Real kappa = P.kappa0 * sl * sl;
        Real drive = P.gbeta_T * (theta_base + P.G * Real(fzc) + P.dT_ref);
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          const Real mc = s_mu[(slot2(C) * NC + i) * NT + tid];
          if constexpr (EXT)
            drive += P.gbeta_c[i] * (P.dcl_ref[i] + P.dceq_dT[0][i] * (theta_base + P.G * Real(fzc)) +
                                     mc * P.inv2A[0]);
          else
            drive += P.gbeta_c[i] * (P.dcl_ref[i] + mc * P.inv2A[0]);
        }
        const Real FB = rho * phl * drive;
        const Real inv = rcp_rn(rho * (Real(1) + Real(0.5) * kappa));
        Real u[3], F[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const Real fb = a == 2 ? FB : Real(0);
          u[a] = (m3[a] + Real(0.5) * (fb + fs[a])) * inv;
          F[a] = fb + fs[a] - rho * kappa * u[a];
          if (a < 2) s_u[(slot2(C) * 2 + a) * NT + tid] = u[a];
        }
        uz_C = u[2];
        if (owner && C >= z0 && C < z0 + ZS && C < P.v_hi) {
          collide<Q>(P, dk, drho, rho, u, F, [&](int k, Real val) {
            const Store v = Codec<Store>::put(val);
            int tx_ = gx + Lat::c(k, 0), ty_ = gy + Lat::c(k, 1), tz_ = C + Lat::c(k, 2), kk = k;
            const bool bx = P.bc[0] == kWall && (tx_ < 0 || tx_ >= nx);
            const bool by = P.bc[1] == kWall && (ty_ < 0 || ty_ >= ny);
            const bool bz = P.bc[2] == kWall && (tz_ < 0 || tz_ >= nz);
            if (bx || by || bz) {  // across a wall the population returns reversed
              kk = Lat::opp(k);
              tx_ = gx;
              ty_ = gy;
              tz_ = C;
            } else {
              tx_ = tx_ < 0 ? tx_ + nx : (tx_ >= nx ? tx_ - nx : tx_);
              ty_ = ty_ < 0 ? ty_ + ny : (ty_ >= ny ? ty_ - ny : ty_);
              tz_ = tz_ < 0 ? tz_ + nz : (tz_ >= nz ? tz_ - nz : tz_);
            }
            f_out[kk * P.plane + (long long)(tz_ - P.zbase) * zst + (long long)ty_ * px + tx_] = v;
          });
        }
      }
      s_chg[slot2(C) * NT + tid] = changed ? 1 : 0;
      s_hl[slot2(C) * NT + tid] = interp_h<NP>(out, 0);
#pragma unroll
      for (int a = 0; a < NP; ++a) pfz_lo[a] = pfz_hi[a];
    }
    __syncthreads();

    // D. solute fluxes of plane M and the update of the owned planes
    const bool doM = M >= z0 - 1 && M <= z0 + ZS - 1;
    const bool outM = doM && M >= z0 && M < P.v_hi;
    // planes M-1 .. M+2 liquid: phi^{n+1} = phi^n = liquid on planes M and
    // M+1, so h_l = 1, M = M0, no antitrapping, chi = 1 / (2 A_l), no obstacles
    const bool lean_d = (liq_hist & 15u) == 15u;
    if (doM) {
      const int fzm = vz(M);
      const bool walls = has_walls;
      // flux between this cell (plane M) and neighbour nb: d normal axis
      auto mu_face = [&](int d, int pB, int nbT, int nbR, int gbd, bool obsB, Real* J) {
        bool closed = (P.bc[d] == kWall && (gbd == 0 || gbd == P.n[d])) || gbd > P.n[d];
        if (!closed && walls && !lean_d) closed = obstacle(P, fx, fy, fzm) || obsB;
#pragma unroll
        for (int i = 0; i < NC; ++i) J[i] = Real(0);
        if (closed) return;
        const int pA = M, A = tid, rA = r2;
        if (lean_d) {
          const Real ua = d == 2 ? uz_M : s_u[(slot2(pA) * 2 + d) * NT + A];
          const Real ub = d == 2 ? uz_C : s_u[(slot2(pB) * 2 + d) * NT + nbT];
          const int fzB = d == 2 ? vz(pB) : fzm;
#pragma unroll
          for (int i = 0; i < NC; ++i) {
            const Real ma = s_mu[(slot2(pA) * NC + i) * NT + A], mb = s_mu[(slot2(pB) * NC + i) * NT + nbT];
            J[i] = liquid_flux(P, ma, mb, ua, ub, ceq_of(0, i, fzm), ceq_of(0, i, fzB));
          }
          return;
        }
        const Real* pnA = s_pn + slot2(pA) * NP * NT;
        const Real* pnB = s_pn + slot2(pB) * NP * NT;
        const Real Mf = Real(0.5) * P.M0 * (pnA[A] + pnB[nbT]);  // plane 0 = liquid
        const Real ua = (d == 2 ? uz_M : s_u[(slot2(pA) * 2 + d) * NT + A]) * s_hl[slot2(pA) * NT + A];
        const Real ub = (d == 2 ? uz_C : s_u[(slot2(pB) * 2 + d) * NT + nbT]) * s_hl[slot2(pB) * NT + nbT];
        const int fzB = d == 2 ? vz(pB) : fzm;  // vertical index of B (ceq(T))
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          const Real ma = s_mu[(slot2(pA) * NC + i) * NT + A], mb = s_mu[(slot2(pB) * NC + i) * NT + nbT];
          J[i] = -Mf * (mb - ma) + Real(0.5) * (ua * (ceq_of(0, i, fzm) + ma * P.inv2A[0]) +
                                                ub * (ceq_of(0, i, fzB) + mb * P.inv2A[0]));
        }
        // the current carries phi_l's face value as a factor of every term: on
        // a face without liquid (grain boundaries inside the solid) it is
        // exactly 0 and skipped
        const Real liq = P.at_eps != Real(0) && (s_chg[slot2(pA) * NT + A] | s_chg[slot2(pB) * NT + nbT])
                             ? Real(0.5) * (PH(pA, 0, rA) + PH(pB, 0, nbR))
                             : Real(0);
        if (liq != Real(0)) {
          Real at[NC];
#pragma unroll
          for (int i = 0; i < NC; ++i) at[i] = Real(0);
#pragma unroll
          for (int a = 1; a < NP; ++a) {
            const Real va = PH(pA, a, rA), vb = PH(pB, a, nbR);
            const Real gn = vb - va;
            Real t1, t2;
            if (d == 2) {
              t1 = Real(0.25) * (PH(pA, a, rA + 1) + PH(pB, a, nbR + 1) - PH(pA, a, rA - 1) - PH(pB, a, nbR - 1));
              t2 = Real(0.25) * (PH(pA, a, rA + W2) + PH(pB, a, nbR + W2) - PH(pA, a, rA - W2) - PH(pB, a, nbR - W2));
            } else {
              const int st = d == 0 ? W2 : 1;
              t1 = Real(0.25) * (PH(pA, a, rA + st) + PH(pB, a, nbR + st) - PH(pA, a, rA - st) - PH(pB, a, nbR - st));
              t2 = Real(0.25) * (PH(pA + 1, a, rA) + PH(pB + 1, a, nbR) - PH(pA - 1, a, rA) - PH(pB - 1, a, nbR));
            }
            const Real g2 = gn * gn + t1 * t1 + t2 * t2;
            if (g2 <= Real(1e-12)) continue;
            const Real nd = liq * gn / sqrt(g2);
            const Real dphi = Real(0.5) * ((pnA[a * NT + A] - va) + (pnB[a * NT + nbT] - vb));
            const Real dinv = P.inv2A[0] - P.inv2A[a];
#pragma unroll
            for (int i = 0; i < NC; ++i) {
              Real dc = (P.ceq[0][i] - P.ceq[a][i]) +
                        Real(0.5) * (s_mu[(slot2(pA) * NC + i) * NT + A] + s_mu[(slot2(pB) * NC + i) * NT + nbT]) * dinv;
              if constexpr (EXT)
                dc += (P.dceq_dT[0][i] - P.dceq_dT[a][i]) * (theta_base + Real(0.5) * P.G * Real(fzm + fzB));
              at[i] += dc * dphi * nd;
            }
          }
#pragma unroll
          for (int i = 0; i < NC; ++i) J[i] -= P.at_eps * at[i];
        }
      };
      // z-face (M, M+1) of this column, for the carry
      {
        const int fzb = vz(M + 1);
        mu_face(2, M + 1, tid, r2, M + 1, walls && !lean_d && obstacle(P, fx, fy, fzb), mz_hi);
      }
      if (M == z0 - 1) {
#pragma unroll
        for (int i = 0; i < NC; ++i) mz_lo[i] = mz_hi[i];
      } else {
        // in-plane faces of plane M
        Real J[NC];
        if (tx < BX - 1) {
          const bool ob = walls && !lean_d && obstacle(P, fold_axis(P, gx + 1, 0), fy, fzm);
          mu_face(0, M, tid + 1, r2 + 1, gx + 1, ob, J);
#pragma unroll
          for (int i = 0; i < NC; ++i) s_flux[(i * 2 + 0) * NT + tid] = J[i];
        }
        if (ty < BY - 1) {
          const bool ob = walls && !lean_d && obstacle(P, fx, fold_axis(P, gy + 1, 1), fzm);
          mu_face(1, M, tid + BX, r2 + W2, gy + 1, ob, J);
#pragma unroll
          for (int i = 0; i < NC; ++i) s_flux[(i * 2 + 1) * NT + tid] = J[i];
        }
      }
    }
    __syncthreads();
    if (outM && M >= z0 && owner) {
      const int fzm = M;  // owned planes lie inside the grid
      const int g = zrow(fzm) + gxy;
      Real po[NP], pn[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        po[a] = PH(M, a, r2);
        pn[a] = s_pn[(slot2(M) * NP + a) * NT + tid];
      }
#pragma unroll
      for (int sidx = 0; sidx < NS; ++sidx) phi_out[sidx * P.plane + g] = pn[NP == 2 ? 1 : sidx];
      out_liq = pure_liquid(pn);
      if (lean_d) {
        // unchanged liquid cell: chi = 1 / (2 A_l); the source is the
        // temperature term alone (extended model)
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          const Real* Jx = s_flux + (i * 2 + 0) * NT;
          const Real* Jy = s_flux + (i * 2 + 1) * NT;
          const Real div = (Jx[tid] - Jx[tid - 1]) + (Jy[tid] - Jy[tid - BX]) + (mz_hi[i] - mz_lo[i]);
          const Real mu = s_mu[(slot2(M) * NC + i) * NT + tid];
          Real src = Real(0);
          if constexpr (EXT) {
#pragma unroll
            for (int a = 0; a < NP; ++a) src -= Real(P.GV) * P.dceq_dT[a][i] * (a == 0 ? Real(1) : Real(0));
          }
          mu_out[i * P.plane + g] = liquid_mu(P, mu, div, src);
        }
      } else if (has_walls && obstacle(P, fx, fy, fzm)) {
#pragma unroll
        for (int i = 0; i < NC; ++i) mu_out[i * P.plane + g] = s_mu[(slot2(M) * NC + i) * NT + tid];
      } else if (!EXT && s_chg[slot2(M) * NT + tid] == 0 && pure_phase<NP>(pn) >= 0) {
        // unchanged pure cell: source term exactly 0, chi = 1 / (2 A_pure)
        const int pa = pure_phase<NP>(pn);
        Real ichi = P.chi_pure[0];
#pragma unroll
        for (int a = 1; a < NP; ++a)
          if (pa == a) ichi = P.chi_pure[a];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          const Real* Jx = s_flux + (i * 2 + 0) * NT;
          const Real* Jy = s_flux + (i * 2 + 1) * NT;
          const Real div = (Jx[tid] - Jx[tid - 1]) + (Jy[tid] - Jy[tid - BX]) + (mz_hi[i] - mz_lo[i]);
          const Real mu = s_mu[(slot2(M) * NC + i) * NT + tid];
          mu_out[i * P.plane + g] = mu + (-div - Real(0)) * ichi;
        }
      } else {
        Real chi = Real(0), hn[NP], ho[NP];
        const bool changed = s_chg[slot2(M) * NT + tid] != 0;
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          hn[a] = interp_h<NP>(pn, a);
          ho[a] = changed ? interp_h<NP>(po, a) : hn[a];
          chi += hn[a] * P.inv2A[a];
        }
        const Real ichi = rcp_rn(chi);
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          const Real* Jx = s_flux + (i * 2 + 0) * NT;
          const Real* Jy = s_flux + (i * 2 + 1) * NT;
          const Real div = (Jx[tid] - Jx[tid - 1]) + (Jy[tid] - Jy[tid - BX]) + (mz_hi[i] - mz_lo[i]);
          const Real mu = s_mu[(slot2(M) * NC + i) * NT + tid];
          Real src = Real(0);
          if (changed) {
#pragma unroll
            for (int a = 0; a < NP; ++a) src += (ceq_of(a, i, fzm) + mu * P.inv2A[a]) * (hn[a] - ho[a]);
          }
          if constexpr (EXT) {
            // -(dT/dt) sum_a (dc_a/dT)_mu h_a^{n+1}, dT/dt = -G V
#pragma unroll
            for (int a = 0; a < NP; ++a) src -= Real(P.GV) * P.dceq_dT[a][i] * hn[a];
          }
          mu_out[i * P.plane + g] = mu + (-div - src) * ichi;
        }
      }
    }
    if (doM && M >= z0) {
#pragma unroll
      for (int i = 0; i < NC; ++i) mz_lo[i] = mz_hi[i];
    }
    if (P.liq_dispatch) {
      // the flag of plane M of this tile (the barrier the loop ends with)
      const bool all = __syncthreads_and(out_liq);
      if (tid == 0 && outM && M >= z0)
        io.flags_out[liquid_flag_index(bx, by, M, gxt, gyt)] = all;
      out_liq = true;
    } else {
      __syncthreads();
    }
  }
}

}  // namespace gpflbm

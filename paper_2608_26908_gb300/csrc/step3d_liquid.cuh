// Liquid tiles of the 3D step.  Away from the solid the phase field is
// pure liquid (phi_l = 1, every other phase 0) in a tile's whole reach, and
// Algorithm 1 reduces there to: phi^{n+1} = phi^n (only one phase is present
// in every 3x3x3 neighbourhood, so it has no rate), the chemical potential
// diffusing with M = D_liq / (2 A_l) and advected by U^n with h_l = 1 and
// chi = 1 / (2 A_l), and the lattice Boltzmann step with phi_l = 1 (no drag,
// the full buoyancy).  liquid_tile advances such tiles with the same
// arithmetic, term for term, as the general path's liquid planes --
// the results are bit-identical -- but without the phase-field machinery,
// so it needs far fewer registers and instructions.
//
// Which tiles are liquid: a flag per tile of the step grid (x tile, y tile,
// z segment) says that every cell the tile owns is pure liquid.  A tile whose
// own flag and its 26 neighbours' flags are set reads only pure liquid (its
// reach is two cells and two planes), so the liquid path takes it;
// otherwise the general path does.  Both write the flags of the tile's new
// state, one per plane.
#pragma once

#include "gpflbm_kernels.cuh"
#include "step3d.cuh"

namespace gpflbm {

template <int NP, int NC, class Real, class Store, int QQ = 19, bool EXT = false>
struct Liquid3D {
  static constexpr int BX = Block3D<Real>::BX, BY = Block3D<Real>::BY, ZS = Block3D<Real>::ZS;
  static constexpr int NT = BX * BY;
  static constexpr int OX = BX - 2, OY = BY - 2;
  static constexpr size_t al(size_t v) { return (v + 15) / 16 * 16; }
  // a ring of three planes of U and mu, and the in-plane solute fluxes of
  // two planes: one barrier a plane (see liquid_tile)
  static constexpr size_t u = 0;                                    // 3 planes x 3 x NT
  static constexpr size_t mu = al(u + sizeof(Real) * 3 * 3 * NT);   // 3 planes x NC x NT
  static constexpr size_t flux = al(mu + sizeof(Real) * 3 * NC * NT);  // 2 planes x 2 x NC x NT
  static constexpr size_t bytes = al(flux + sizeof(Real) * 2 * 2 * NC * NT);
};

// The liquid path for one tile (coordinates as for general_tile).
template <int NP, int NC, class Real, class Store, int QQ, bool EXT>
__device__ __forceinline__ void liquid_tile(const DevParams<Real>& P, const Step3DIO& io, int bx, int by, int bz,
                                            int gxt, int gyt) {
  using S = Liquid3D<NP, NC, Real, Store, QQ, EXT>;
  using Lat = Lattice<QQ>;
  constexpr int BX = S::BX, BY = S::BY, ZS = S::ZS, NT = S::NT, Q = QQ;
  constexpr int NS = PhiStore<NP>::NS;
  extern __shared__ __align__(16) unsigned char smem[];
  Real* s_u = reinterpret_cast<Real*>(smem + S::u);
  Real* s_mu = reinterpret_cast<Real*>(smem + S::mu);
  Real* s_flux = reinterpret_cast<Real*>(smem + S::flux);

  const Real* __restrict__ mu_in = static_cast<const Real*>(io.mu_in);
  const Store* __restrict__ f_in = static_cast<const Store*>(io.f_in);
  Real* __restrict__ phi_out = static_cast<Real*>(io.phi_out);
  Real* __restrict__ mu_out = static_cast<Real*>(io.mu_out);
  Store* __restrict__ f_out = static_cast<Store*>(io.f_out);

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2], px = P.px;
  const int zst = px * ny;
  const int x0 = bx * S::OX, y0 = by * S::OY, z0 = P.v_lo + bz * ZS;
  const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
  const bool inner_xy = x0 >= 2 && x0 - 2 + BX + 2 <= nx && y0 >= 2 && y0 - 2 + BY + 2 <= ny;
  const int fx = inner_xy ? gx : fold_axis(P, gx, 0);
  const int fy = inner_xy ? gy : fold_axis(P, gy, 1);
  const int gxy = fy * px + fx;
  const bool owner = tx >= 1 && tx <= BX - 2 && ty >= 1 && ty <= BY - 2 && gx < nx && gy < ny;
  const double t_now = io.clock_in[0];
  if (bx == 0 && by == 0 && bz == 0 && tid == 0) io.clock_out[0] = t_now + 1.0;
  const Real theta_base = Real(P.theta0) - Real(P.GV) * Real(t_now);
  auto ceq_of = [&](int a, int i, int v) -> Real {
    if constexpr (EXT)
      return fma_rn(P.dceq_dT[a][i], fma_rn(P.G, Real(v), theta_base), P.ceq[a][i]);
    else
      return P.ceq[a][i];
  };
  auto vz = [&](int v) {
    const int f = fold_axis(P, v, 2);
    return f < P.v_lo - 2 ? P.v_lo - 2 : (f > P.v_hi + 1 ? P.v_hi + 1 : f);
  };
  auto zrow = [&](int fz) { return (fz - P.zbase) * zst; };
  // the segment and its two halo planes lie inside the grid: no folding and
  // no closed z-face (in-plane faces of an inner tile are never closed)
  const bool zin = z0 >= 1 && z0 + ZS <= nz - 1;
  auto vzi = [&](int v) { return zin ? v : vz(v); };

  // solute z-face fluxes of this column: (M-1, M) carried, (M, M+1) new
  Real mz_lo[NC], mz_hi[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) mz_lo[i] = mz_hi[i] = Real(0);

  // Ring slots of planes M and C = M + 1.  One barrier a plane: the in-plane
  // fluxes of a plane are formed in the iteration that produced its U and
  // mu, into one half of a double buffer, and read by the next iteration's
  // update; three slots of U and mu, so that the slot B overwrites held the
  // plane three back, which no thread reads after the previous barrier.
  int sM = 2, sC = 0;
  for (int C = z0 - 1; C <= z0 + ZS; ++C) {
    const int M = C - 1;
    // B. moments, U and (owned planes) collision + push, plane C
    {
      const int fzc = vzi(C);
      const int gi = zrow(fzc) + gxy;
      Real mu[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        mu[i] = (mu_in + i * P.plane)[gi];
        s_mu[(sC * NC + i) * NT + tid] = mu[i];
      }
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
      // the general path's arithmetic with phi_l = 1 (the same helpers)
      const Real drive = buoyancy_drive<NC, EXT>(P, fma_rn(P.G, Real(fzc), theta_base), mu);
      Real u[3], F[3];
      force_velocity<3>(P, rho, Real(1), drive, m3, u, F);
#pragma unroll
      for (int a = 0; a < 3; ++a) s_u[(sC * 3 + a) * NT + tid] = u[a];
      if (owner && C >= z0 && C < z0 + ZS && C < P.v_hi) {
        const bool inner_z = C >= 1 && C + 1 < nz;
        if (inner_xy && inner_z) {
          Store* const fo = f_out + gi;
          collide<Q>(P, dk, drho, rho, u, F, [&](int k, Real val) { at_bytes(fo, P.f_to[k]) = Codec<Store>::put(val); });
        } else {
          const PushAxis X = push_axis(gx, nx, P.bc[0] == kWall, 1);
          const PushAxis Y = push_axis(gy, ny, P.bc[1] == kWall, px);
          const PushAxis Z = push_axis(C, nz, P.bc[2] == kWall, zst);
          collide<Q>(P, dk, drho, rho, u, F, [&](int k, Real val) {
            push_store<Lat>(f_out, P.plane, gi, k, Codec<Store>::put(val), X, Y, Z);
          });
        }
      }
    }
    __syncthreads();
    // D. solute fluxes (every plane M-1 .. C+1 liquid: M = M0, h_l = 1).
    // face between this cell in plane pA (slot sA) and nbT in plane pB (slot sB)
    auto face = [&](int d, int pA, int sA, int pB, int sB, int nbT, int gbd, Real* J) {
      const bool open = d == 2 ? zin : inner_xy;
      const bool closed = !open && ((P.bc[d] == kWall && (gbd == 0 || gbd == P.n[d])) || gbd > P.n[d]);
#pragma unroll
      for (int i = 0; i < NC; ++i) J[i] = Real(0);
      if (closed) return;
      const int fzA = vzi(pA);
      const Real ua = s_u[(sA * 3 + d) * NT + tid], ub = s_u[(sB * 3 + d) * NT + nbT];
      const int fzB = d == 2 ? vzi(pB) : fzA;
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        const Real ma = s_mu[(sA * NC + i) * NT + tid], mb = s_mu[(sB * NC + i) * NT + nbT];
        J[i] = liquid_flux(P, ma, mb, ua, ub, ceq_of(0, i, fzA), ceq_of(0, i, fzB));
      }
    };
    // the z-face (M, C) of this column
    const bool doM = M >= z0 - 1 && M <= z0 + ZS - 1;
    if (doM) {
      face(2, M, sM, C, sC, tid, C, mz_hi);
      if (M == z0 - 1) {
#pragma unroll
        for (int i = 0; i < NC; ++i) mz_lo[i] = mz_hi[i];
      }
    }
    // the update of plane M: its in-plane fluxes (formed last iteration) and
    // its two z-faces
    if (doM && M >= z0 && M < P.v_hi && owner) {
      const Real* fl = s_flux + (M & 1) * 2 * NC * NT;
      const int g = zrow(M) + gxy;
#pragma unroll
      for (int sidx = 0; sidx < NS; ++sidx)
        phi_out[sidx * P.plane + g] = (NP != 2 && sidx == 0) ? Real(1) : Real(0);
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        const Real* Jx = fl + (i * 2 + 0) * NT;
        const Real* Jy = fl + (i * 2 + 1) * NT;
        const Real div = (Jx[tid] - Jx[tid - 1]) + (Jy[tid] - Jy[tid - BX]) + (mz_hi[i] - mz_lo[i]);
        const Real mu = s_mu[(sM * NC + i) * NT + tid];
        Real src = Real(0);
        if constexpr (EXT) {
#pragma unroll
          for (int a = 0; a < NP; ++a) src -= Real(P.GV) * P.dceq_dT[a][i] * (a == 0 ? Real(1) : Real(0));
        }
        mu_out[i * P.plane + g] = liquid_mu(P, mu, div, src);
      }
    }
    if (doM && M >= z0) {
#pragma unroll
      for (int i = 0; i < NC; ++i) mz_lo[i] = mz_hi[i];
    }
    // the in-plane fluxes of plane C, for its update in the next iteration
    if (C >= z0 && C <= z0 + ZS - 1) {
      Real* fl = s_flux + (C & 1) * 2 * NC * NT;
      Real J[NC];
      if (tx < BX - 1) {
        face(0, C, sC, C, sC, tid + 1, gx + 1, J);
#pragma unroll
        for (int i = 0; i < NC; ++i) fl[(i * 2 + 0) * NT + tid] = J[i];
      }
      if (ty < BY - 1) {
        face(1, C, sC, C, sC, tid + BX, gy + 1, J);
#pragma unroll
        for (int i = 0; i < NC; ++i) fl[(i * 2 + 1) * NT + tid] = J[i];
      }
    }
    sM = sC;
    sC = sC == 2 ? 0 : sC + 1;
  }
  if (tid < ZS && z0 + tid < P.v_hi) io.flags_out[liquid_flag_index(bx, by, z0 + tid, gxt, gyt)] = 1;
}

// The step kernels.  Where both paths fit 64 registers (FP32 arithmetic on
// D3Q19: two CTAs share an SM either way) and the general path is that of
// two phases (Step3D::ONE_LAUNCH), one launch takes every tile: its
// grid holds the tiling twice, z blocks 0 .. gzt-1 the general pass and
// gzt .. 2 gzt-1 the liquid pass, and a CTA returns unless its tile's flags
// pick its pass.  CTAs start in block order, so the general tiles, the slow
// ones, start first and the liquid tiles fill the SMs as they finish
// instead of waiting for the last general tile.  Elsewhere (FP64, D3Q27:
// the general path needs more registers than the liquid one, and one kernel
// would hold the liquid tiles to its occupancy; three or four phases: its
// shared memory, see ONE_LAUNCH) step3d_kernel takes the general tiles and
// step3d_liquid_kernel, launched after it, the others.
template <int NP, int NC, class Real, class Store, bool SHRINK = false, int QQ = 19, bool EXT = false>
__global__ void __launch_bounds__(Step3D<NP, NC, Real, Store, QQ>::NT, Step3D<NP, NC, Real, Store, QQ>::MIN_CTAS)
    step3d_kernel(const DevParams<Real> P, const Step3DIO io) {
  using S = Step3D<NP, NC, Real, Store, QQ>;
  constexpr int ZS = S::ZS;
  const int gxt = gridDim.x, gyt = gridDim.y, gzt = (P.v_hi - P.v_lo + ZS - 1) / ZS;
  const int bx = blockIdx.x, by = blockIdx.y;
  const bool liquid_pass = S::ONE_LAUNCH && (int)blockIdx.z >= gzt;
  const int bz = liquid_pass ? (int)blockIdx.z - gzt : (int)blockIdx.z;
  if (P.liq_dispatch && liquid_reach<ZS>(P, io.flags_in, bx, by, P.v_lo + bz * ZS, gxt, gyt) != liquid_pass) return;
  if constexpr (S::ONE_LAUNCH) {
    if (liquid_pass) {
      liquid_tile<NP, NC, Real, Store, QQ, EXT>(P, io, bx, by, bz, gxt, gyt);
      return;
    }
  }
  general_tile<NP, NC, Real, Store, SHRINK, QQ, EXT>(P, io, bx, by, bz, gxt, gyt);
}

template <int NP, int NC, class Real, class Store, int QQ = 19, bool EXT = false>
__global__ void __launch_bounds__(Liquid3D<NP, NC, Real, Store, QQ, EXT>::NT, 2)
    step3d_liquid_kernel(const DevParams<Real> P, const Step3DIO io) {
  constexpr int ZS = Liquid3D<NP, NC, Real, Store, QQ, EXT>::ZS;
  if (!liquid_reach<ZS>(P, io.flags_in, blockIdx.x, blockIdx.y, P.v_lo + blockIdx.z * ZS, gridDim.x, gridDim.y))
    return;
  liquid_tile<NP, NC, Real, Store, QQ, EXT>(P, io, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y);
}

// The liquid flags of a state (after a load or a frame shift): one CTA per
// xy tile and plane, the flag set when every cell the tile owns in the plane
// is pure liquid.
template <int NP, class Real>
__global__ void liquid_flags_kernel(const DevParams<Real> P, const Real* __restrict__ phi,
                                    unsigned char* __restrict__ flags) {
  constexpr int BX = Block3D<Real>::BX, BY = Block3D<Real>::BY;
  constexpr int OX = BX - 2, OY = BY - 2;
  const int x0 = blockIdx.x * OX, y0 = blockIdx.y * OY, z = P.v_lo + blockIdx.z;
  const int wx = min(OX, P.n[0] - x0), wy = min(OY, P.n[1] - y0);
  const int zst = P.px * P.n[1];
  bool liq = true;
  for (int c = threadIdx.x; c < wx * wy; c += blockDim.x) {
    const int x = x0 + c % wx, y = y0 + c / wx;
    Real v[NP];
    load_phases<NP>(phi, (long long)(z - P.zbase) * zst + (long long)y * P.px + x, P.plane, v);
    bool p = v[0] == Real(1);
#pragma unroll
    for (int a = 1; a < NP; ++a) p = p && v[a] == Real(0);
    liq = liq && p;
  }
  liq = __syncthreads_and(liq);
  if (threadIdx.x == 0) flags[liquid_flag_index(blockIdx.x, blockIdx.y, z, gridDim.x, gridDim.y)] = liq;
}

}  // namespace gpflbm

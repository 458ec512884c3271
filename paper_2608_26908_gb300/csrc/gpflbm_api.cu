// C-ABI of the coupled Grand-Potential phase-field / lattice-Boltzmann step
// (declared and documented in include/gpflbm.h).  Host logic only: argument
// checks, workspace layout, parameter preparation, CUDA-graph replay of the
// step, and dispatch to the kernel table of the problem's configuration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "adjoint_ops.h"
#include "gpflbm.h"
#include "gpflbm_ops.cuh"

using gpflbm::DevParams;
using gpflbm::Ops;

namespace {

constexpr size_t kAlign = 256;
constexpr double kPi = 3.14159265358979323846;
constexpr int kChunk = 16;  // steps per replayed CUDA graph

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
  size_t phi[2], mu[2], f[2], stage, clock, partial, red, flags[2];
  size_t total;
};

}  // namespace

struct gpflbm_s {
  gpflbm_grid grid;
  gpflbm_params params;
  int NP, NC, Q, D;
  long long cells, plane;
  int px;  // padded row pitch (elements)
  const Ops* ops;
  const Ops* ops_ext;  // the same configuration, extended model (tilt, ceq(T))
  Layout lay;
  unsigned char* ws;
  bool owns_ws;
  int cur;            // buffer holding the current state
  long long t;        // step counter of the current state
  bool has_state;
  cudaStream_t capture;
  // adjoint: the stream that recomputes segments, and its events
  cudaStream_t aux;
  cudaEvent_t ev_fwd, ev_aux_end, ev_rec[2], ev_adj[2];
  cudaGraphExec_t chunk_graph[2];
  cudaGraphExec_t pair_graph[2];
  // Asynchronous loads (GPFLBM_ASYNC from device or pinned sources) write the
  // idle buffer on their own stream, so that they overlap the read-only calls
  // (fields, deviations, invariants) that precede them on the caller's
  // stream.  ev_mark is recorded on the caller's stream after every call that
  // writes or reads both buffers (mut counts those calls; marked is the count
  // at the last record); a load waits for it, and the caller's stream waits
  // for the load.  Every entry point other than the read-only ones bumps mut.
  cudaStream_t xfer;
  cudaEvent_t ev_mark, ev_loaded;
  unsigned long long mut, marked;
  // device parameters in the arithmetic type (only one is used)
  DevParams<double> pd;
  DevParams<float> pf;
  gpflbm::InvParams inv;
  std::string err;
  // Slab of the vertical axis (3D, gpflbm_create_slab): the handle owns the
  // planes v_lo .. v_hi - 1 of the grid, and its buffers hold two halo planes
  // on each side (hz = 2; 0 for a whole grid).  The step runs in the grid's
  // coordinates (pd, pf); the state exchange, fields and totals see the
  // owned planes as a grid of their own (xd, xf).  halo_fresh: the halo
  // planes next to a neighbouring slab (lower, upper) were written since the
  // last step.
  bool slab;
  int v_lo, v_hi, hz;
  long long zst;  // elements per vertical plane of the buffers (px * ny)
  bool halo_fresh[2];
  DevParams<double> xd;
  DevParams<float> xf;
};

namespace {

gpflbm_status fail(gpflbm_t h, gpflbm_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

gpflbm_status cuda_fail(gpflbm_t h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, GPFLBM_ERR_CUDA, m);
}

// The kernel table the time steps use: the extended model's when a pair of
// the problem's phases has a nonzero tilt or an equilibrium composition
// depends on temperature.
const Ops* stepper(gpflbm_t h) { return h->pf.tilted || h->pf.tdep ? h->ops_ext : h->ops; }

// Record the caller's stream's progress for asynchronous loads, once per
// run of read-only calls (see gpflbm_s::ev_mark).
void mark(gpflbm_t h, cudaStream_t s) {
  if (h->xfer && h->marked != h->mut) {
    cudaEventRecord(h->ev_mark, s);
    h->marked = h->mut;
  }
}

const Ops* find_ops(int D, int lattice, int precision, int NP, int NC, bool ext) {
  using namespace gpflbm;
#define GPFLBM_PICK(NAME) return ext ? NAME##_ext(NP, NC) : NAME(NP, NC)
  if (lattice == GPFLBM_D3Q27) {
    switch (precision) {
      case GPFLBM_FP64: GPFLBM_PICK(ops_d3q27_fp64);
      case GPFLBM_FP32: GPFLBM_PICK(ops_d3q27_fp32);
    }
    return nullptr;
  }
  if (D == 2) {
    switch (precision) {
      case GPFLBM_FP64: GPFLBM_PICK(ops_d2_fp64);
      case GPFLBM_FP32: GPFLBM_PICK(ops_d2_fp32);
      case GPFLBM_FP32_F16STORE: GPFLBM_PICK(ops_d2_f16);
      case GPFLBM_FP32_BF16STORE: GPFLBM_PICK(ops_d2_bf16);
    }
  } else {
    switch (precision) {
      case GPFLBM_FP64: GPFLBM_PICK(ops_d3_fp64);
      case GPFLBM_FP32: GPFLBM_PICK(ops_d3_fp32);
      case GPFLBM_FP32_F16STORE: GPFLBM_PICK(ops_d3_f16);
      case GPFLBM_FP32_BF16STORE: GPFLBM_PICK(ops_d3_bf16);
    }
  }
#undef GPFLBM_PICK
  return nullptr;
}

// Validates the grid; fills D and the kernel table.
gpflbm_status check_grid(const gpflbm_grid* g, int NP, int NC, int* D, const Ops** ops,
                         std::string* why) {
  if (!g) {
    *why = "grid is NULL";
    return GPFLBM_ERR_ARG;
  }
  if (g->nx < 3 || g->ny < 3 || g->nz < 1 || (g->nz > 1 && g->nz < 3)) {
    *why = "grid needs nx, ny >= 3 and nz == 1 or nz >= 3";
    return GPFLBM_ERR_ARG;
  }
  const long long cells = (long long)g->nx * g->ny * g->nz;
  if (cells > (1LL << 31) - 1024) {
    *why = "grid has more than 2^31 cells";
    return GPFLBM_ERR_ARG;
  }
  *D = g->nz == 1 ? 2 : 3;
  if ((*D == 2 && g->lattice != GPFLBM_D2Q9) ||
      (*D == 3 && g->lattice != GPFLBM_D3Q19 && g->lattice != GPFLBM_D3Q27)) {
    *why = "lattice must be D2Q9 for nz == 1 and D3Q19 or D3Q27 otherwise";
    return GPFLBM_ERR_UNSUPPORTED;
  }
  for (int a = 0; a < 3; ++a) {
    if (g->bc[a] != GPFLBM_PERIODIC && g->bc[a] != GPFLBM_WALL) {
      *why = "bc must be GPFLBM_PERIODIC or GPFLBM_WALL";
      return GPFLBM_ERR_ARG;
    }
    const int n = a == 0 ? g->nx : (a == 1 ? g->ny : g->nz);
    if (g->wall_rows[a] < 0 || (a < *D && 2 * g->wall_rows[a] >= n) || (a >= *D && g->wall_rows[a] != 0)) {
      *why = "wall_rows out of range";
      return GPFLBM_ERR_ARG;
    }
  }
  {
    // kernels index a cell within a field plane with 32 bits
    const long long px = ((long long)g->nx + 7) / 8 * 8;
    const long long nz = *D == 3 ? g->nz : 1;
    if (px * g->ny * nz + 64 > 0x7fffffffLL) {
      *why = "a field plane must hold fewer than 2^31 cells";
      return GPFLBM_ERR_UNSUPPORTED;
    }
  }
  if (g->precision < GPFLBM_FP64 || g->precision > GPFLBM_FP32_BF16STORE) {
    *why = "unknown precision";
    return GPFLBM_ERR_ARG;
  }
  if (NP < 2 || NP > GPFLBM_MAX_PHASES || NC < 1 || NC > GPFLBM_MAX_SOLUTES) {
    *why = "n_phases must be 2..4 and n_components 1..2";
    return GPFLBM_ERR_UNSUPPORTED;
  }
  *ops = find_ops(*D, g->lattice, g->precision, NP, NC, false);
  if (!*ops) {
    *why = "configuration not built";
    return GPFLBM_ERR_UNSUPPORTED;
  }
  return GPFLBM_OK;
}

// xy tiles of the 3D step grid (an upper bound over the arithmetic types)
// times planes: one liquid flag each.
long long step_tiles(const gpflbm_grid* g, int nz_own) {
  using F = gpflbm::Block3D<float>;
  using Dd = gpflbm::Block3D<double>;
  const long long ox = F::BX - 2 < Dd::BX - 2 ? F::BX - 2 : Dd::BX - 2;
  const long long oy = F::BY - 2 < Dd::BY - 2 ? F::BY - 2 : Dd::BY - 2;
  return ((g->nx + ox - 1) / ox) * ((g->ny + oy - 1) / oy) * nz_own;
}

Layout make_layout(const Ops* ops, long long cells, long long plane, long long tiles) {
  (void)cells;
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = round_up(off + bytes, kAlign);
    return at;
  };
  for (int i = 0; i < 2; ++i) L.phi[i] = take(ops->stored_phi_planes * plane * ops->real_size);
  for (int i = 0; i < 2; ++i) L.mu[i] = take(ops->NC * plane * ops->real_size);
  for (int i = 0; i < 2; ++i) L.f[i] = take(ops->Q * plane * ops->store_size);
  L.stage = take(ops->Q * plane * ops->real_size);
  L.clock = take(2 * sizeof(double));
  L.partial = take(gpflbm::kRedMaxBlocks * (ops->NC + 3) * sizeof(double));
  L.red = take((ops->NC + 3) * sizeof(double));
  for (int i = 0; i < 2; ++i) L.flags[i] = take((size_t)tiles);
  L.total = off;
  return L;
}

// Velocity c_k of the lattice with Q populations (D2Q9, D3Q19, D3Q27).
void lattice_velocity(int Q, int k, int* c) {
  for (int a = 0; a < 3; ++a)
    c[a] = Q == 9 ? (a < 2 ? gpflbm::Lattice<9>::c(k, a) : 0)
                  : (Q == 19 ? gpflbm::Lattice<19>::c(k, a) : gpflbm::Lattice<27>::c(k, a));
}

template <class Real>
void fill_params(gpflbm_t h, DevParams<Real>& P) {
  const gpflbm_params& p = h->params;
  std::memset(&P, 0, sizeof(P));
  P.n[0] = h->grid.nx;
  P.n[1] = h->grid.ny;
  P.n[2] = h->D == 3 ? h->grid.nz : 1;
  for (int a = 0; a < 3; ++a) {
    P.bc[a] = a < h->D ? h->grid.bc[a] : GPFLBM_PERIODIC;
    P.wall[a] = a < h->D ? h->grid.wall_rows[a] : 0;
  }
  P.px = h->px;
  P.plane = h->plane;
  P.eps = (Real)p.eps;
  P.mob_eps = (Real)(1.0 / (p.tau_phi * p.eps));
  P.obst = (Real)(16.0 / (kPi * kPi * p.eps));
  for (int a = 0; a < 4; ++a) {
    for (int b = 0; b < 4; ++b) {
      P.gamma[a][b] = (Real)p.gamma[a][b];
      P.delta[a][b] = (Real)p.delta[a][b];
      if (a < h->NP && b < h->NP && a != b && P.delta[a][b] != Real(0)) P.aniso = 1;
    }
    P.inv2A[a] = (Real)(1.0 / (2.0 * p.A[a]));
    P.inv4A[a] = (Real)(1.0 / (4.0 * p.A[a]));
    P.chi_pure[a] = Real(1) / P.inv2A[a];  // IEEE division in Real, as on the device
    P.eta[a] = a < h->NP ? (Real)p.eta_rho[a] : Real(0);
    if (P.eta[a] != Real(0)) P.shrink = 1;
    for (int b = 0; b < 4; ++b) {
      const double th = a < h->NP && b < h->NP && a != b ? p.tilt[a][b] : 0.0;
      P.tilt_c[a][b] = (Real)std::cos(th);
      P.tilt_s[a][b] = (Real)std::sin(th);
      if (th != 0.0) P.tilted = P.aniso = 1;
    }
    for (int i = 0; i < 2; ++i) {
      const double k = a < h->NP && i < h->NC ? p.dceq_dT[a][i] : 0.0;
      P.dceq_dT[a][i] = (Real)k;
      if (k != 0.0) P.tdep = 1;
    }
    for (int i = 0; i < 2; ++i) P.ceq[a][i] = (Real)p.ceq[a][i];
    P.S[a] = (Real)p.S[a];
  }
  for (int i = 0; i < 2; ++i) P.dcl_ref[i] = (Real)(p.ceq[0][i] - p.c_ref[i]);
  P.M0 = (Real)(p.D_liq / (2.0 * p.A[0]));
  P.at_eps = (Real)(p.a_at * p.eps);
  const double nu = (p.tau_f - 0.5) / 3.0;
  P.kappa0 = (Real)(2.0 * nu * p.h_drag / (p.W0 * p.W0));
  for (int i = 0; i < 2; ++i) P.gbeta_c[i] = (Real)p.gbeta_c[i];
  P.gbeta_T = (Real)p.gbeta_T;
  P.dT_ref = (Real)(p.T_E - p.T_ref);
  P.G = (Real)p.G;
  P.inv_tau_f = (Real)(1.0 / p.tau_f);
  P.force_pre = (Real)(1.0 - 0.5 / p.tau_f);
  P.q_floor = (Real)p.q_floor;
  P.theta0 = -p.undercool - p.G * p.v0;
  P.GV = p.G * p.V;
  P.v_lo = 0;
  P.v_hi = h->D == 3 ? h->grid.nz : h->grid.ny;
  P.zbase = 0;
  // population byte offsets: a cell's own k, and where its collided k lands
  const long long es = (long long)h->ops->store_size, zst = (long long)h->px * h->grid.ny;
  for (int k = 0; k < h->ops->Q; ++k) {
    int c[3];
    lattice_velocity(h->ops->Q, k, c);
    P.f_at[k] = (long long)k * h->plane * es;
    P.f_to[k] = ((long long)k * h->plane + c[0] + (long long)c[1] * h->px + (long long)c[2] * zst) * es;
  }
}

gpflbm_status check_params(const gpflbm_params* p, int NP, std::string* why) {
  if (!p) {
    *why = "params is NULL";
    return GPFLBM_ERR_ARG;
  }
  if (!(p->tau_f > 0.5) || !(p->tau_phi > 0.0) || !(p->eps > 0.0) || !(p->W0 > 0.0)) {
    *why = "need tau_f > 1/2, tau_phi > 0, eps > 0, W0 > 0";
    return GPFLBM_ERR_ARG;
  }
  for (int a = 0; a < NP; ++a)
    if (!(p->A[a] > 0.0)) {
      *why = "need A_a > 0 for every phase";
      return GPFLBM_ERR_ARG;
    }
  for (int a = 0; a < NP; ++a)
    if (!std::isfinite(p->eta_rho[a])) {
      *why = "eta_rho must be finite";
      return GPFLBM_ERR_ARG;
    }
  for (int a = 0; a < NP; ++a)
    for (int b = 0; b < NP; ++b)
      if (a != b && (!std::isfinite(p->tilt[a][b]) || p->tilt[a][b] != p->tilt[b][a])) {
        *why = "tilt must be finite and symmetric";
        return GPFLBM_ERR_ARG;
      }
  for (int a = 0; a < NP; ++a)
    for (int i = 0; i < 2; ++i)
      if (!std::isfinite(p->dceq_dT[a][i])) {
        *why = "dceq_dT must be finite";
        return GPFLBM_ERR_ARG;
      }
  if (!(p->D_liq >= 0.0) || !(p->q_floor >= 0.0)) {
    *why = "need D_liq >= 0 and q_floor >= 0";
    return GPFLBM_ERR_ARG;
  }
  return GPFLBM_OK;
}

template <class Real>
void slab_views(gpflbm_t h, DevParams<Real>& P, DevParams<Real>& X) {
  if (!h->slab) return;
  P.v_lo = h->v_lo;
  P.v_hi = h->v_hi;
  P.zbase = h->v_lo - h->hz;
  X = P;
  X.n[2] = h->v_hi - h->v_lo;
  X.theta0 = P.theta0 + (double)P.G * h->v_lo;  // T at owned plane v is T at grid plane v_lo + v
  X.v_lo = 0;
  X.v_hi = X.n[2];
  X.zbase = 0;
}

// Liquid tiles take the lean kernel in 3D, except on slabs (their halo
// planes come from another handle), with shrinkage or obstacle rows, and
// where a periodic x or y axis ends in a tile of one cell (a tile's reach
// would then wrap past its neighbour tiles; planes are flagged one by one).
bool liquid_dispatch(gpflbm_t h) {
  if (h->D != 3 || h->slab || h->pf.shrink) return false;
  const gpflbm_grid& g = h->grid;
  if (g.wall_rows[0] | g.wall_rows[1] | g.wall_rows[2]) return false;
  const bool fp64 = g.precision == GPFLBM_FP64;
  const int o[2] = {(fp64 ? gpflbm::Block3D<double>::BX : gpflbm::Block3D<float>::BX) - 2,
                    (fp64 ? gpflbm::Block3D<double>::BY : gpflbm::Block3D<float>::BY) - 2};
  const int n[2] = {g.nx, g.ny};
  for (int a = 0; a < 2; ++a)
    if (g.bc[a] == GPFLBM_PERIODIC && n[a] % o[a] == 1) return false;
  return true;
}

void set_device_params(gpflbm_t h) {
  fill_params(h, h->pd);
  fill_params(h, h->pf);
  const int liq = liquid_dispatch(h) ? 1 : 0;
  h->pd.liq_dispatch = h->pf.liq_dispatch = liq;
  slab_views(h, h->pd, h->xd);
  slab_views(h, h->pf, h->xf);
  h->inv.cells = h->cells;
  h->inv.plane = h->plane;
  h->inv.nx = h->grid.nx;
  h->inv.px = h->px;
  h->inv.vlayer = h->D == 3 ? (long long)h->grid.nx * h->grid.ny : h->grid.nx;
  h->inv.G = h->params.G;
  h->inv.tdep = 0;
  for (int a = 0; a < 4; ++a) {
    for (int i = 0; i < 2; ++i) {
      h->inv.ceq[a][i] = h->params.ceq[a][i];
      h->inv.dceq_dT[a][i] = a < h->NP && i < h->NC ? h->params.dceq_dT[a][i] : 0.0;
      if (h->inv.dceq_dT[a][i] != 0.0) h->inv.tdep = 1;
    }
    h->inv.inv2A[a] = 1.0 / (2.0 * h->params.A[a]);
  }
}

const void* dev_params(gpflbm_t h) {
  return h->grid.precision == GPFLBM_FP64 ? (const void*)&h->pd : (const void*)&h->pf;
}

// Parameters of the state-exchange, field and totals kernels: the owned
// planes as a grid of their own (a whole grid: the step's parameters).
const void* xparams(gpflbm_t h) {
  if (!h->slab) return dev_params(h);
  return h->grid.precision == GPFLBM_FP64 ? (const void*)&h->xd : (const void*)&h->xf;
}

void* at(gpflbm_t h, size_t off) { return h->ws + off; }

// First owned plane of a field buffer at workspace offset `off` whose
// elements are `esize` bytes (the buffer start for a whole grid).
void* own(gpflbm_t h, size_t off, size_t esize) {
  return h->ws + off + (size_t)h->hz * (size_t)h->zst * esize;
}

gpflbm::StepIO step_io(gpflbm_t h, int from) {
  gpflbm::StepIO io;
  io.phi_in = at(h, h->lay.phi[from]);
  io.phi_out = at(h, h->lay.phi[1 - from]);
  io.mu_in = at(h, h->lay.mu[from]);
  io.mu_out = at(h, h->lay.mu[1 - from]);
  io.f_in = at(h, h->lay.f[from]);
  io.f_out = at(h, h->lay.f[1 - from]);
  io.clock_in = reinterpret_cast<const double*>(at(h, h->lay.clock)) + from;
  io.clock_out = reinterpret_cast<double*>(at(h, h->lay.clock)) + 1 - from;
  io.flags_in = static_cast<const unsigned char*>(at(h, h->lay.flags[from]));
  io.flags_out = static_cast<unsigned char*>(at(h, h->lay.flags[1 - from]));
  return io;
}

// The device address of a host buffer the GPU can read and write directly:
// pinned or registered host memory, mapped into the device's address space
// (over NVLink-C2C on a Grace-Blackwell node the kernels stream it at link
// speed).  nullptr for pageable memory, which has to be staged.
void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer is not an error here
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

__global__ void set_clock_kernel(double* clock, double t) {
  clock[0] = t;
  clock[1] = t;
}

void drop_graphs(gpflbm_t h) {
  for (int i = 0; i < 2; ++i) {
    if (h->chunk_graph[i]) cudaGraphExecDestroy(h->chunk_graph[i]);
    if (h->pair_graph[i]) cudaGraphExecDestroy(h->pair_graph[i]);
    h->chunk_graph[i] = h->pair_graph[i] = nullptr;
  }
}

// Liquid flags of the tiles of state buffer `buf` (3D with the liquid
// dispatch; nothing otherwise).
cudaError_t classify(gpflbm_t h, int buf, cudaStream_t s) {
  if (!h->pf.liq_dispatch) return cudaSuccess;
  return h->ops->classify(dev_params(h), at(h, h->lay.phi[buf]),
                          static_cast<unsigned char*>(at(h, h->lay.flags[buf])), s);
}

// A slab steps only with both halos next to a neighbouring slab written
// since its last step; the step then uses them up.
gpflbm_status slab_ready(gpflbm_t h, const char* what) {
  if (!h->slab) return GPFLBM_OK;
  const bool lo = h->v_lo > 0, hi = h->v_hi < h->grid.nz;
  if ((lo && !h->halo_fresh[0]) || (hi && !h->halo_fresh[1]))
    return fail(h, GPFLBM_ERR_STATE, std::string(what) + ": exchange the slab's halo planes before each step");
  h->halo_fresh[0] = h->halo_fresh[1] = false;
  return GPFLBM_OK;
}

// The fixed-order totals of the current state's owned cells into `red`.
cudaError_t run_invariants(gpflbm_t h, double* partial, int blocks, double* red, cudaStream_t s) {
  const double theta0 = h->slab ? h->xd.theta0 : h->pd.theta0;
  h->inv.theta_t = theta0 - h->pd.GV * (double)h->t;
  const size_t rs = h->ops->real_size;
  return h->ops->invariants(h->inv, own(h, h->lay.phi[h->cur], rs), own(h, h->lay.mu[h->cur], rs),
                            own(h, h->lay.f[h->cur], h->ops->store_size), partial, blocks, red, s);
}

// Captures `steps` consecutive steps starting from buffer `from`.
gpflbm_status capture(gpflbm_t h, int from, int steps, cudaGraphExec_t* out) {
  cudaError_t e = cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
  int b = from;
  cudaError_t le = cudaSuccess;
  for (int s = 0; s < steps; ++s) {
    le = stepper(h)->step(dev_params(h), step_io(h, b), h->capture);
    if (le != cudaSuccess) break;
    b = 1 - b;
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(h->capture, &graph);
  if (le != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(h, le, "step launch during capture");
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  return GPFLBM_OK;
}

}  // namespace

extern "C" {

gpflbm_status gpflbm_workspace_bytes(const gpflbm_grid* grid, int n_phases, int n_components,
                                     size_t* bytes) {
  int D;
  const Ops* ops;
  std::string why;
  if (!bytes) return GPFLBM_ERR_ARG;
  gpflbm_status st = check_grid(grid, n_phases, n_components, &D, &ops, &why);
  if (st != GPFLBM_OK) return st;
  const long long cells = (long long)grid->nx * grid->ny * grid->nz;
  const size_t px = round_up(grid->nx, 8);
  *bytes = make_layout(ops, cells, (long long)round_up(px * grid->ny * grid->nz, 64),
                       step_tiles(grid, grid->nz)).total;
  return GPFLBM_OK;
}

}  // extern "C"

namespace {

// Planes v_begin .. v_begin + v_count - 1 of the vertical axis of a 3D grid
// as a slab: walls on that axis, no obstacle rows on it, at least two planes.
gpflbm_status check_slab(const gpflbm_grid* g, int D, int v_begin, int v_count, std::string* why) {
  if (D != 3) {
    *why = "slabs: 3D grids only";
    return GPFLBM_ERR_UNSUPPORTED;
  }
  if (g->bc[2] != GPFLBM_WALL || g->wall_rows[2] != 0) {
    *why = "slabs: the vertical axis needs walls and no obstacle rows";
    return GPFLBM_ERR_UNSUPPORTED;
  }
  if (v_begin < 0 || v_count < 2 || (long long)v_begin + v_count > g->nz) {
    *why = "slabs: need 0 <= v_begin, v_count >= 2, v_begin + v_count <= nz";
    return GPFLBM_ERR_ARG;
  }
  return GPFLBM_OK;
}

// Planes held by a slab's buffers: its own and two halo planes on each side.
constexpr int kHalo = 2;

gpflbm_status create_impl(const gpflbm_grid* grid, int n_phases, int n_components,
                          const gpflbm_params* params, void* workspace, size_t workspace_bytes,
                          bool slab, int v_begin, int v_count, gpflbm_t* out) {
  if (!out) return GPFLBM_ERR_ARG;
  *out = nullptr;
  int D;
  const Ops* ops;
  std::string why;
  gpflbm_status st = check_grid(grid, n_phases, n_components, &D, &ops, &why);
  if (st == GPFLBM_OK && slab) st = check_slab(grid, D, v_begin, v_count, &why);
  if (st != GPFLBM_OK) {
    std::fprintf(stderr, "gpflbm_create: %s\n", why.c_str());
    return st;
  }
  st = check_params(params, n_phases, &why);
  if (st == GPFLBM_OK && slab) {
    for (int a = 0; a < n_phases; ++a)
      if (params->eta_rho[a] != 0.0) {
        why = "slabs: shrinkage is not supported";
        st = GPFLBM_ERR_UNSUPPORTED;
      }
  }
  if (st != GPFLBM_OK) {
    std::fprintf(stderr, "gpflbm_create: %s\n", why.c_str());
    return st;
  }
  gpflbm_t h = new (std::nothrow) gpflbm_s();
  if (!h) return GPFLBM_ERR_OOM;
  h->grid = *grid;
  h->params = *params;
  h->NP = n_phases;
  h->NC = n_components;
  h->D = D;
  h->Q = ops->Q;
  h->ops = ops;
  h->ops_ext = find_ops(D, grid->lattice, grid->precision, n_phases, n_components, true);
  h->slab = slab;
  h->v_lo = slab ? v_begin : 0;
  h->v_hi = slab ? v_begin + v_count : (D == 3 ? grid->nz : grid->ny);
  h->hz = slab ? kHalo : 0;
  const int nz_own = slab ? v_count : grid->nz;
  h->cells = (long long)grid->nx * grid->ny * nz_own;
  h->px = (int)round_up(grid->nx, 8);
  h->zst = (long long)h->px * grid->ny;
  h->plane = (long long)round_up((size_t)h->zst * (nz_own + 2 * h->hz), 64);
  h->lay = make_layout(ops, h->cells, h->plane, step_tiles(grid, nz_own));
  h->cur = 0;
  h->t = 0;
  h->has_state = false;
  if (workspace) {
    if (workspace_bytes < h->lay.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) {
      const gpflbm_status bad = workspace_bytes < h->lay.total ? GPFLBM_ERR_OOM : GPFLBM_ERR_ARG;
      delete h;
      std::fprintf(stderr, "gpflbm_create: workspace too small or not 256-byte aligned\n");
      return bad;
    }
    h->ws = static_cast<unsigned char*>(workspace);
    h->owns_ws = false;
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, h->lay.total);
    if (e != cudaSuccess) {
      delete h;
      return GPFLBM_ERR_OOM;
    }
    h->ws = static_cast<unsigned char*>(p);
    h->owns_ws = true;
  }
  cudaError_t e = h->ops->configure();
  if (e == cudaSuccess) e = h->ops_ext->configure();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "gpflbm_create: %s\n", cudaGetErrorString(e));
    if (h->owns_ws) cudaFree(h->ws);
    delete h;
    return GPFLBM_ERR_CUDA;
  }
  e = cudaMemset(h->ws, 0, h->lay.total);  // padding cells stay finite
  if (e != cudaSuccess) {
    std::fprintf(stderr, "gpflbm_create: %s\n", cudaGetErrorString(e));
    gpflbm_destroy(h);
    return GPFLBM_ERR_CUDA;
  }
  set_device_params(h);
  *out = h;
  return GPFLBM_OK;
}

}  // namespace

extern "C" {

gpflbm_status gpflbm_create(const gpflbm_grid* grid, int n_phases, int n_components,
                            const gpflbm_params* params, void* workspace, size_t workspace_bytes,
                            gpflbm_t* out) {
  return create_impl(grid, n_phases, n_components, params, workspace, workspace_bytes, false, 0, 0, out);
}

gpflbm_status gpflbm_slab_workspace_bytes(const gpflbm_grid* grid, int v_begin, int v_count, int n_phases,
                                          int n_components, size_t* bytes) {
  int D;
  const Ops* ops;
  std::string why;
  if (!bytes) return GPFLBM_ERR_ARG;
  gpflbm_status st = check_grid(grid, n_phases, n_components, &D, &ops, &why);
  if (st == GPFLBM_OK) st = check_slab(grid, D, v_begin, v_count, &why);
  if (st != GPFLBM_OK) return st;
  const size_t px = round_up(grid->nx, 8);
  const long long cells = (long long)grid->nx * grid->ny * v_count;
  *bytes = make_layout(ops, cells, (long long)round_up(px * grid->ny * (v_count + 2 * kHalo), 64),
                       step_tiles(grid, v_count)).total;
  return GPFLBM_OK;
}

gpflbm_status gpflbm_create_slab(const gpflbm_grid* grid, int v_begin, int v_count, int n_phases,
                                 int n_components, const gpflbm_params* params, void* workspace,
                                 size_t workspace_bytes, gpflbm_t* out) {
  return create_impl(grid, n_phases, n_components, params, workspace, workspace_bytes, true, v_begin,
                     v_count, out);
}

gpflbm_status gpflbm_set_params(gpflbm_t h, const gpflbm_params* params) {
  if (!h) return GPFLBM_ERR_ARG;
  std::string why;
  gpflbm_status st = check_params(params, h->NP, &why);
  if (st != GPFLBM_OK) return fail(h, st, why);
  if (h->slab)
    for (int a = 0; a < h->NP; ++a)
      if (params->eta_rho[a] != 0.0) return fail(h, GPFLBM_ERR_UNSUPPORTED, "set_params: no shrinkage on a slab");
  h->params = *params;
  const int had = h->pf.liq_dispatch;
  set_device_params(h);
  drop_graphs(h);  // parameters are baked into captured launches
  ++h->mut;
  if (h->has_state && h->pf.liq_dispatch && !had) {
    // the flags were not kept while every tile took the general path
    cudaError_t e = classify(h, h->cur, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_params: liquid tiles");
  }
  return GPFLBM_OK;
}

gpflbm_status gpflbm_set_state(gpflbm_t h, const void* phi, const void* mu, const void* f,
                               int src_is_device, long long t0, void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  if (!phi || !mu) return fail(h, GPFLBM_ERR_ARG, "set_state: phi and mu are required");
  if (src_is_device & ~(GPFLBM_ON_DEVICE | GPFLBM_ASYNC))
    return fail(h, GPFLBM_ERR_ARG, "set_state: unknown flag");
  const bool on_device = (src_is_device & GPFLBM_ON_DEVICE) != 0;
  const bool async = (src_is_device & GPFLBM_ASYNC) != 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t rs = h->ops->real_size;
  const size_t n = (size_t)h->cells;
  const void* sp = phi;
  const void* sm = mu;
  const void* sf = f;
  const size_t ss = h->ops->store_size;
  void* phi_d = own(h, h->lay.phi[h->cur], rs);
  void* mu_d = own(h, h->lay.mu[h->cur], rs);
  void* f_d = own(h, h->lay.f[h->cur], ss);
  cudaError_t e;
  bool staged = false;
  if (!on_device) {
    // pinned host sources are read by the load kernels in place
    void* mp = mapped_host(phi);
    void* mm = mapped_host(mu);
    void* mf = f ? mapped_host(f) : nullptr;
    if (mp && mm && (!f || mf)) {
      sp = mp;
      sm = mm;
      sf = mf;
    } else {
      staged = true;
    }
  }
  if (staged) {
    // stage through the idle buffers: phi in the stage area, mu in the idle
    // mu buffer, f in the stage area after phi has been converted
    unsigned char* stage = static_cast<unsigned char*>(at(h, h->lay.stage));
    e = cudaMemcpyAsync(stage, phi, h->NP * n * rs, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state: copy phi");
    e = h->ops->load(xparams(h), stage, nullptr, nullptr, phi_d, mu_d, f_d, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state: load phi");
    e = cudaMemcpyAsync(stage, mu, h->NC * n * rs, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state: copy mu");
    e = h->ops->load(xparams(h), nullptr, stage, nullptr, phi_d, mu_d, f_d, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state: load mu");
    sp = sm = nullptr;
    if (f) {
      e = cudaMemcpyAsync(stage, f, h->Q * n * rs, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "set_state: copy f");
      sf = stage;
    }
  }
  double* clk = reinterpret_cast<double*>(at(h, h->lay.clock));
  if (!staged && async && h->has_state) {
    // Load the idle buffer on the library's transfer stream once the caller's
    // stream has finished the last call that used both buffers, so that the
    // load overlaps the read-only calls queued since (a write-back of the
    // current state over the host link runs beside the next state's load);
    // the caller's stream then waits for the load.
    if (!h->xfer) {
      e = cudaStreamCreateWithFlags(&h->xfer, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_mark, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_loaded, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        if (h->xfer) cudaStreamDestroy(h->xfer);
        h->xfer = nullptr;
        return cuda_fail(h, e, "set_state: transfer stream");
      }
      h->marked = h->mut + 1;  // nothing recorded yet
    }
    mark(h, s);
    const int to = 1 - h->cur;
    e = cudaStreamWaitEvent(h->xfer, h->ev_mark, 0);
    if (e == cudaSuccess)
      e = h->ops->load_state(xparams(h), sp, sm, sf, own(h, h->lay.phi[to], rs), own(h, h->lay.mu[to], rs),
                             own(h, h->lay.f[to], ss), clk + to, nullptr, (double)t0, h->xfer);
    if (e == cudaSuccess) e = classify(h, to, h->xfer);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_loaded, h->xfer);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_loaded, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state: load");
    h->cur = to;
    h->t = t0;
    h->halo_fresh[0] = h->halo_fresh[1] = false;
    ++h->mut;
    return GPFLBM_OK;
  }
  if (staged) {
    // (the load launcher always rewrites f: from sf, or the fluid at rest)
    e = h->ops->load(xparams(h), sp, sm, sf, phi_d, mu_d, f_d, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state: load");
    set_clock_kernel<<<1, 1, 0, s>>>(clk, (double)t0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state: clock");
  } else {
    // device or pinned sources: every plane and the counters in one launch
    e = h->ops->load_state(xparams(h), sp, sm, sf, phi_d, mu_d, f_d, clk, clk + 1, (double)t0, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state: load");
  }
  e = classify(h, h->cur, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state: liquid tiles");
  if (staged || !async) {
    e = cudaStreamSynchronize(s);  // host sources must outlive the copies and loads
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state: synchronize");
  }
  h->t = t0;
  h->has_state = true;
  h->halo_fresh[0] = h->halo_fresh[1] = false;
  ++h->mut;
  return GPFLBM_OK;
}

gpflbm_status gpflbm_step(gpflbm_t h, int n_steps, void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  if (n_steps < 0) return fail(h, GPFLBM_ERR_ARG, "step: n_steps < 0");
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, "step: no state loaded");
  if (h->slab && n_steps > 1) return fail(h, GPFLBM_ERR_ARG, "step: a slab steps once per halo exchange");
  if (n_steps > 0) {
    gpflbm_status st = slab_ready(h, "step");
    if (st != GPFLBM_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ++h->mut;
  int left = n_steps;
  while (left > 0) {
    cudaError_t e;
    if (left >= kChunk) {
      if (!h->chunk_graph[h->cur]) {
        gpflbm_status st = capture(h, h->cur, kChunk, &h->chunk_graph[h->cur]);
        if (st != GPFLBM_OK) return st;
      }
      e = cudaGraphLaunch(h->chunk_graph[h->cur], s);
      left -= kChunk;  // even: the state returns to the same buffer
    } else if (left >= 2) {
      if (!h->pair_graph[h->cur]) {
        gpflbm_status st = capture(h, h->cur, 2, &h->pair_graph[h->cur]);
        if (st != GPFLBM_OK) return st;
      }
      e = cudaGraphLaunch(h->pair_graph[h->cur], s);
      left -= 2;
    } else {
      e = stepper(h)->step(dev_params(h), step_io(h, h->cur), s);
      h->cur = 1 - h->cur;
      left -= 1;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
  }
  h->t += n_steps;
  return GPFLBM_OK;
}

gpflbm_status gpflbm_shift_frame(gpflbm_t h, int rows, void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  if (h->slab) return fail(h, GPFLBM_ERR_UNSUPPORTED, "shift_frame: not on a slab");
  const int ax = h->D == 3 ? 2 : 1;
  const int nv = ax == 2 ? h->grid.nz : h->grid.ny;
  if (rows < 0 || rows >= nv) return fail(h, GPFLBM_ERR_ARG, "shift_frame: need 0 <= rows < n_vertical");
  if (h->grid.wall_rows[ax] != 0)
    return fail(h, GPFLBM_ERR_UNSUPPORTED, "shift_frame: obstacle rows on the vertical axis");
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, "shift_frame: no state loaded");
  if (rows == 0) return GPFLBM_OK;
  ++h->mut;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long layer = ax == 2 ? (long long)h->px * h->grid.ny : h->px;
  const long long n = layer * nv;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  const int from = h->cur, to = 1 - h->cur;
  auto move = [&](size_t src_off, size_t dst_off, int planes, size_t word) {
    const void* a = at(h, src_off);
    void* b = at(h, dst_off);
    switch (word) {
      case 2:
        gpflbm::shift_frame_kernel<unsigned short><<<blocks, threads, 0, s>>>(
            static_cast<const unsigned short*>(a), static_cast<unsigned short*>(b), planes, h->plane, n,
            layer, nv, rows);
        break;
      case 4:
        gpflbm::shift_frame_kernel<unsigned int><<<blocks, threads, 0, s>>>(
            static_cast<const unsigned int*>(a), static_cast<unsigned int*>(b), planes, h->plane, n, layer,
            nv, rows);
        break;
      default:
        gpflbm::shift_frame_kernel<unsigned long long><<<blocks, threads, 0, s>>>(
            static_cast<const unsigned long long*>(a), static_cast<unsigned long long*>(b), planes,
            h->plane, n, layer, nv, rows);
    }
    return cudaGetLastError();
  };
  cudaError_t e = move(h->lay.phi[from], h->lay.phi[to], h->ops->stored_phi_planes, h->ops->real_size);
  if (e == cudaSuccess) e = move(h->lay.mu[from], h->lay.mu[to], h->NC, h->ops->real_size);
  if (e == cudaSuccess) e = move(h->lay.f[from], h->lay.f[to], h->Q, h->ops->store_size);
  if (e == cudaSuccess) {
    double* clk = reinterpret_cast<double*>(at(h, h->lay.clock));
    e = cudaMemcpyAsync(clk + to, clk + from, sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "shift_frame");
  h->cur = to;
  h->params.v0 -= rows;
  set_device_params(h);
  e = classify(h, to, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "shift_frame: liquid tiles");
  drop_graphs(h);  // v0 is baked into captured launches
  return GPFLBM_OK;
}

gpflbm_status gpflbm_step_timed(gpflbm_t h, void* const* events, void* stream) {
  if (!h || !events || !events[0] || !events[1])
    return fail(h, GPFLBM_ERR_ARG, "step_timed: two events are required");
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, "step_timed: no state loaded");
  {
    gpflbm_status st = slab_ready(h, "step_timed");
    if (st != GPFLBM_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ++h->mut;
  const gpflbm::StepIO io = step_io(h, h->cur);
  cudaError_t e = cudaEventRecord(static_cast<cudaEvent_t>(events[0]), s);
  if (e == cudaSuccess) e = stepper(h)->step(dev_params(h), io, s);
  if (e == cudaSuccess) e = cudaEventRecord(static_cast<cudaEvent_t>(events[1]), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "step_timed");
  h->cur = 1 - h->cur;
  h->t += 1;
  return GPFLBM_OK;
}

gpflbm_status gpflbm_get_fields(gpflbm_t h, unsigned field_mask, void* const* dst,
                                int dst_is_device, void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, "get_fields: no state loaded");
  if (field_mask & ~63u) return fail(h, GPFLBM_ERR_ARG, "get_fields: unknown field bit");
  if (field_mask && !dst) return fail(h, GPFLBM_ERR_ARG, "get_fields: dst is NULL");
  if (dst_is_device & ~(GPFLBM_ON_DEVICE | GPFLBM_ASYNC))
    return fail(h, GPFLBM_ERR_ARG, "get_fields: unknown flag");
  const bool on_device = (dst_is_device & GPFLBM_ON_DEVICE) != 0;
  const bool async = (dst_is_device & GPFLBM_ASYNC) != 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mark(h, s);  // read-only: a later asynchronous load may overlap it
  const size_t rs = h->ops->real_size;
  const size_t n = (size_t)h->cells;
  const int planes[6] = {h->NP, h->NC, h->NC, h->Q, 1, h->D};
  gpflbm::FieldsIO base;
  std::memset(&base, 0, sizeof(base));
  base.phi = own(h, h->lay.phi[h->cur], rs);
  base.mu = own(h, h->lay.mu[h->cur], rs);
  base.f = own(h, h->lay.f[h->cur], h->ops->store_size);
  base.clock = reinterpret_cast<const double*>(at(h, h->lay.clock)) + h->cur;
  // device and pinned host destinations are written by one launch; pageable
  // host destinations go through the stage area one field at a time
  gpflbm::FieldsIO direct = base;
  void** outs_direct[6] = {&direct.o_phi, &direct.o_mu, &direct.o_c, &direct.o_f, &direct.o_rho, &direct.o_u};
  void* staged_dst[6] = {};
  bool any_direct = false;
  int slot = 0;
  for (int bit = 0; bit < 6; ++bit) {
    if (!(field_mask & (1u << bit))) continue;
    void* d = dst[slot++];
    if (!d) return fail(h, GPFLBM_ERR_ARG, "get_fields: a destination is NULL");
    void* m = on_device ? d : mapped_host(d);
    if (m) {
      *outs_direct[bit] = m;
      any_direct = true;
    } else {
      staged_dst[bit] = d;
    }
  }
  cudaError_t e;
  if (any_direct) {
    e = h->ops->fields(xparams(h), direct, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_fields: kernel");
  }
  for (int bit = 0; bit < 6; ++bit) {
    if (!staged_dst[bit]) continue;
    void* target = at(h, h->lay.stage);
    gpflbm::FieldsIO io = base;
    void** outs[6] = {&io.o_phi, &io.o_mu, &io.o_c, &io.o_f, &io.o_rho, &io.o_u};
    *outs[bit] = target;
    e = h->ops->fields(xparams(h), io, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_fields: kernel");
    e = cudaMemcpyAsync(staged_dst[bit], target, planes[bit] * n * rs, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_fields: copy");
    e = cudaStreamSynchronize(s);  // the stage area is reused by the next field
    if (e != cudaSuccess) return cuda_fail(h, e, "get_fields: synchronize");
  }
  bool any_staged = false;
  for (int bit = 0; bit < 6; ++bit) any_staged = any_staged || staged_dst[bit] != nullptr;
  if (!on_device && (any_staged || !async)) {
    e = cudaStreamSynchronize(s);  // host destinations are complete on return
    if (e != cudaSuccess) return cuda_fail(h, e, "get_fields: synchronize");
  }
  return GPFLBM_OK;
}

gpflbm_status gpflbm_get_deviations(gpflbm_t h, void* dst, int dst_is_device, void* stream) {
  if (!h || !dst) return GPFLBM_ERR_ARG;
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, "get_deviations: no state loaded");
  if (dst_is_device & ~(GPFLBM_ON_DEVICE | GPFLBM_ASYNC))
    return fail(h, GPFLBM_ERR_ARG, "get_deviations: unknown flag");
  const bool on_device = (dst_is_device & GPFLBM_ON_DEVICE) != 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mark(h, s);  // read-only
  void* target = on_device ? dst : at(h, h->lay.stage);
  gpflbm::FieldsIO io;
  std::memset(&io, 0, sizeof(io));
  io.phi = own(h, h->lay.phi[h->cur], h->ops->real_size);
  io.mu = own(h, h->lay.mu[h->cur], h->ops->real_size);
  io.f = own(h, h->lay.f[h->cur], h->ops->store_size);
  io.clock = reinterpret_cast<const double*>(at(h, h->lay.clock)) + h->cur;
  io.o_dev = target;
  cudaError_t e = h->ops->fields(xparams(h), io, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_deviations: kernel");
  if (!on_device) {
    e = cudaMemcpyAsync(dst, target, h->Q * (size_t)h->cells * h->ops->real_size,
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_deviations: copy");
  }
  return GPFLBM_OK;
}

gpflbm_status gpflbm_invariants(gpflbm_t h, double* mass, double* solute, double* solid_frac,
                                void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, "invariants: no state loaded");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mark(h, s);  // read-only
  const long long want = (h->cells + gpflbm::kRedThreads - 1) / gpflbm::kRedThreads;
  const int blocks = (int)(want < gpflbm::kRedMaxBlocks ? want : gpflbm::kRedMaxBlocks);
  double* partial = reinterpret_cast<double*>(at(h, h->lay.partial));
  double* red = reinterpret_cast<double*>(at(h, h->lay.red));
  cudaError_t e = run_invariants(h, partial, blocks, red, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "invariants: kernel");
  double out[GPFLBM_MAX_SOLUTES + 3];
  e = cudaMemcpyAsync(out, red, (h->NC + 3) * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "invariants: copy");
  if (mass) *mass = out[0] + (double)h->cells;
  if (solute)
    for (int i = 0; i < h->NC; ++i) solute[i] = out[1 + i];
  if (solid_frac) *solid_frac = out[h->NC + 1] / (double)h->cells;
  if (out[h->NC + 2] != 0.0)
    return fail(h, GPFLBM_ERR_NONFINITE, "invariants: NaN or Inf in the state");
  return GPFLBM_OK;
}

}  // extern "C"

namespace gpflbm {
// Whole vertical planes between a slab's state buffers and a halo message:
// segment j moves words[j] 16-byte words from src[j] to dst[j] (blockIdx.y
// picks the segment; a grid-stride loop over its words in x).
constexpr int kHaloMaxSegs = 48;
struct HaloCopy {
  const uint4* src[kHaloMaxSegs];
  uint4* dst[kHaloMaxSegs];
  long long words[kHaloMaxSegs];
};

__global__ void halo_copy_kernel(const HaloCopy c) {
  const int j = blockIdx.y;
  const uint4* __restrict__ src = c.src[j];
  uint4* __restrict__ dst = c.dst[j];
  const long long n = c.words[j];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}
}  // namespace gpflbm

namespace {

// Bytes of one halo message: two planes of phi (every stored component) and
// one plane of mu and of the stored populations.
size_t halo_message_bytes(gpflbm_t h) {
  const size_t rs = h->ops->real_size, ss = h->ops->store_size, z = (size_t)h->zst;
  return (2 * (size_t)h->ops->stored_phi_planes + h->NC) * z * rs + (size_t)h->Q * z * ss;
}

// Copies the planes a neighbour on `side` (0 below, 1 above) needs into msg
// (pack), or the neighbour's planes from msg into this slab's halo (unpack).
// Message: phi of the lower plane (every stored component), phi of the upper
// plane, mu, the stored populations; planes in the buffers' own layout.
gpflbm_status halo_copy(gpflbm_t h, int side, unsigned char* msg, bool pack, cudaStream_t s) {
  const int phi_first = pack ? (side == 0 ? h->v_lo : h->v_hi - 2) : (side == 0 ? h->v_lo - 2 : h->v_hi);
  const int one = pack ? (side == 0 ? h->v_lo : h->v_hi - 1) : (side == 0 ? h->v_lo - 1 : h->v_hi);
  const size_t rs = h->ops->real_size, ss = h->ops->store_size, z = (size_t)h->zst;
  auto local = [&](int g) { return (size_t)(g - (h->v_lo - h->hz)); };
  gpflbm::HaloCopy c;
  int n = 0;
  size_t off = 0;
  auto add = [&](unsigned char* plane, size_t bytes) {
    unsigned char* a = pack ? plane : msg + off;
    unsigned char* b = pack ? msg + off : plane;
    c.src[n] = reinterpret_cast<const uint4*>(a);
    c.dst[n] = reinterpret_cast<uint4*>(b);
    c.words[n] = (long long)(bytes / 16);
    ++n;
    off += bytes;
  };
  unsigned char* phi = static_cast<unsigned char*>(at(h, h->lay.phi[h->cur]));
  unsigned char* mu = static_cast<unsigned char*>(at(h, h->lay.mu[h->cur]));
  unsigned char* f = static_cast<unsigned char*>(at(h, h->lay.f[h->cur]));
  for (int l = 0; l < 2; ++l)
    for (int a = 0; a < h->ops->stored_phi_planes; ++a)
      add(phi + ((size_t)a * h->plane + local(phi_first + l) * z) * rs, z * rs);
  for (int i = 0; i < h->NC; ++i) add(mu + ((size_t)i * h->plane + local(one) * z) * rs, z * rs);
  for (int k = 0; k < h->Q; ++k) add(f + ((size_t)k * h->plane + local(one) * z) * ss, z * ss);
  long long most = 0;
  for (int j = 0; j < n; ++j) most = c.words[j] > most ? c.words[j] : most;
  const unsigned bx = (unsigned)((most + 255) / 256 < 64 ? (most + 255) / 256 : 64);
  gpflbm::halo_copy_kernel<<<dim3(bx, n), 256, 0, s>>>(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, pack ? "halo_pack" : "halo_unpack");
  return GPFLBM_OK;
}

gpflbm_status halo_check(gpflbm_t h, int side, const void* msg, const char* what) {
  if (!h->slab) return fail(h, GPFLBM_ERR_UNSUPPORTED, std::string(what) + ": the handle is not a slab");
  if (side != 0 && side != 1) return fail(h, GPFLBM_ERR_ARG, std::string(what) + ": side must be 0 or 1");
  if ((side == 0 && h->v_lo == 0) || (side == 1 && h->v_hi == h->grid.nz))
    return fail(h, GPFLBM_ERR_ARG, std::string(what) + ": no neighbouring slab on that side (a wall)");
  if (!msg || (reinterpret_cast<uintptr_t>(msg) & 15u) != 0)
    return fail(h, GPFLBM_ERR_ARG, std::string(what) + ": message must be 16-byte aligned device memory");
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, std::string(what) + ": no state loaded");
  return GPFLBM_OK;
}

}  // namespace

extern "C" {

gpflbm_status gpflbm_halo_bytes(gpflbm_t h, size_t* bytes) {
  if (!h || !bytes) return GPFLBM_ERR_ARG;
  if (!h->slab) return fail(h, GPFLBM_ERR_UNSUPPORTED, "halo_bytes: the handle is not a slab");
  *bytes = halo_message_bytes(h);
  return GPFLBM_OK;
}

gpflbm_status gpflbm_halo_pack(gpflbm_t h, int side, void* msg, void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  gpflbm_status st = halo_check(h, side, msg, "halo_pack");
  if (st != GPFLBM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mark(h, s);  // read-only
  return halo_copy(h, side, static_cast<unsigned char*>(msg), true, s);
}

gpflbm_status gpflbm_halo_unpack(gpflbm_t h, int side, const void* msg, void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  gpflbm_status st = halo_check(h, side, msg, "halo_unpack");
  if (st != GPFLBM_OK) return st;
  ++h->mut;
  st = halo_copy(h, side, static_cast<unsigned char*>(const_cast<void*>(msg)), false,
                 static_cast<cudaStream_t>(stream));
  if (st == GPFLBM_OK) h->halo_fresh[side] = true;
  return st;
}

gpflbm_status gpflbm_step_launches(gpflbm_t h, int* launches) {
  if (!h || !launches) return GPFLBM_ERR_ARG;
  *launches = h->pf.liq_dispatch ? stepper(h)->liquid_step_launches : 1;
  return GPFLBM_OK;
}

gpflbm_status gpflbm_time(gpflbm_t h, long long* t) {
  if (!h || !t) return GPFLBM_ERR_ARG;
  *t = h->t;
  return GPFLBM_OK;
}

const char* gpflbm_last_error(gpflbm_t h) { return h ? h->err.c_str() : "null handle"; }

void gpflbm_destroy(gpflbm_t h) {
  if (!h) return;
  drop_graphs(h);
  if (h->capture) cudaStreamDestroy(h->capture);
  if (h->xfer) {
    // an asynchronous load may still write the workspace, which the caller
    // may free once this returns
    cudaStreamSynchronize(h->xfer);
    cudaStreamDestroy(h->xfer);
    cudaEventDestroy(h->ev_mark);
    cudaEventDestroy(h->ev_loaded);
  }
  if (h->aux) {
    cudaStreamDestroy(h->aux);
    cudaEventDestroy(h->ev_fwd);
    cudaEventDestroy(h->ev_aux_end);
    for (int i = 0; i < 2; ++i) {
      cudaEventDestroy(h->ev_rec[i]);
      cudaEventDestroy(h->ev_adj[i]);
    }
  }
  if (h->owns_ws) cudaFree(h->ws);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Conservation totals without any allocation.
//
// Some callers cannot allocate device memory when they need the totals: a
// process whose device memory is already reserved by another framework's
// caching allocator, or a watchdog or logging hook that must not touch the
// allocator while a simulation runs.  This variant of gpflbm_invariants keeps
// its reduction scratch (the per-block partial sums and the final totals) in
// a file-scope device array instead of the handle's workspace, so it needs
// neither cudaMalloc nor workspace beyond the state itself.
//
// The array is kNoAllocDoubles doubles (80 KB) and lives on every GPU that
// loads the library until the process exits.  Blocks of 256 threads each sum
// up to 8192 cells, so at most 2048 blocks fit: grids of more than
// 16,777,216 cells are rejected.  Calls share the array; every slot a call
// reads is written earlier by the same call, so nothing needs clearing, but
// two calls that overlap on the GPU (on different streams or devices sharing
// a handle) race on it.  The device address of the array is looked up once
// per device, on the first call made with that device current; that first
// call should come before any stream capture.
namespace {
constexpr int kNoAllocThreads = gpflbm::kRedThreads;
constexpr long long kNoAllocCellsPerBlock = kNoAllocThreads * 32LL;
constexpr int kNoAllocMaxBlocks = 2048;
constexpr int kNoAllocValues = GPFLBM_MAX_SOLUTES + 3;
constexpr size_t kNoAllocDoubles = (size_t)(kNoAllocMaxBlocks + 1) * kNoAllocValues;
constexpr int kNoAllocMaxDevices = 64;
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace {
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device.
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" gpflbm_status gpflbm_invariants_noalloc(gpflbm_t h, double* mass, double* solute,
                                                   double* solid_frac, void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  const long long blocks = (h->cells + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock;
  if (blocks > kNoAllocMaxBlocks) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "invariants_noalloc: %lld cells exceed the static scratch limit of %lld cells",
                  h->cells, (long long)kNoAllocMaxBlocks * kNoAllocCellsPerBlock);
    return fail(h, GPFLBM_ERR_ARG, msg);
  }
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, "invariants_noalloc: no state loaded");
  double* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return cuda_fail(h, e, "invariants_noalloc: cudaGetSymbolAddress");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mark(h, s);  // read-only
  double* partial = scratch;
  double* red = scratch + (size_t)kNoAllocMaxBlocks * kNoAllocValues;
  e = run_invariants(h, partial, (int)blocks, red, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "invariants_noalloc: kernel");
  double out[kNoAllocValues];
  e = cudaMemcpyAsync(out, red, (h->NC + 3) * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "invariants_noalloc: copy");
  if (mass) *mass = out[0] + (double)h->cells;
  if (solute)
    for (int i = 0; i < h->NC; ++i) solute[i] = out[1 + i];
  if (solid_frac) *solid_frac = out[h->NC + 1] / (double)h->cells;
  if (out[h->NC + 2] != 0.0)
    return fail(h, GPFLBM_ERR_NONFINITE, "invariants_noalloc: NaN or Inf in the state");
  return GPFLBM_OK;
}

// ---------------------------------------------------------------------------
// Adjoint with checkpointing (2D, two phases, one solute).
//
// Workspace: ceil(H/K) checkpoints, two sets of K segment states, one clock
// per stored state, two adjoint states (ping-pong), 3 FP64 accumulator
// planes and the reduction partials.  A stored state is 11 planes: phi_1,
// mu, f - w (9).
//
// Schedule.  The forward pass steps from checkpoint to checkpoint through
// the segment slots (segment c: ckpt[c] -> seg[c % 2][0] -> ... ->
// ckpt[c+1]); the last segment stays in its slots, so the backward pass
// starts without a recompute.  Every earlier segment is recomputed from its
// checkpoint (K - 1 steps) on a second stream into the other set of slots
// while the adjoint steps of the segment after it run: the two kernels
// share the SMs and fill each other's idle tail.  Events order a recompute
// after the adjoint that last read its slots, and an adjoint after its
// recompute.  Forward steps in total: H + (ceil(H/K) - 1) (K - 1).

namespace {

struct AdjLayout {
  size_t state;  // bytes of one stored state
  int n_ck, K;
  size_t ckpt, seg[2], clk, lam[2], gacc, partial, tip, total;
};

AdjLayout adj_layout(gpflbm_t h, int H, int K) {
  AdjLayout L;
  const size_t pl = (size_t)h->plane * h->ops->real_size;
  L.K = K < H ? K : H;
  L.n_ck = (H + L.K - 1) / L.K;
  L.state = 11 * pl;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t a = off;
    off = round_up(off + bytes, kAlign);
    return a;
  };
  L.ckpt = take((size_t)L.n_ck * L.state);
  for (int i = 0; i < 2; ++i) L.seg[i] = take((size_t)L.K * L.state);
  L.clk = take((size_t)(L.n_ck + 2 * L.K) * sizeof(double));
  for (int i = 0; i < 2; ++i) L.lam[i] = take(L.state);
  L.gacc = take(3 * (size_t)h->plane * sizeof(double));
  L.partial = take(4 * (size_t)gpflbm::kRedMaxBlocks * sizeof(double));
  L.tip = take(sizeof(double));
  L.total = off;
  return L;
}

gpflbm_status adj_check(gpflbm_t h, int H, int K) {
  const int prec = h->grid.precision;
  if (h->D != 2 || h->NP != 2 || h->NC != 1 || (prec != GPFLBM_FP64 && prec != GPFLBM_FP32) ||
      h->pf.shrink || h->pd.shrink)
    return fail(h, GPFLBM_ERR_UNSUPPORTED,
                "adjoint: built for 2D, two phases, one solute, in FP64 or FP32, without shrinkage");
  if (H < 1 || K < 1) return fail(h, GPFLBM_ERR_ARG, "adjoint: need horizon >= 1 and ckpt_every >= 1");
  return GPFLBM_OK;
}

// With obj the adjoint seed is dJ/dS of the objective of the final state;
// with seed (obj NULL) it is the 11 given planes (a linear functional of
// the final state), and grad receives all 11 planes of lambda^{t0}.
gpflbm_status adjoint_run(gpflbm_t h, const gpflbm_objective* obj, int H, const AdjLayout& L,
                          unsigned char* ws, double* J, double* dparams, void* dmu0, int dst_is_device,
                          cudaStream_t s, const void* seed = nullptr, void* grad = nullptr) {
  const gpflbm::AdjOps* A = gpflbm::adjoint_ops(h->grid.precision == GPFLBM_FP64);
  const void* P = dev_params(h);
  const size_t pl = (size_t)h->plane * h->ops->real_size;
  const int K = L.K, n_ck = L.n_ck;
  double* clk = reinterpret_cast<double*>(ws + L.clk);
  cudaError_t e = A->configure();
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: configure");
  if (!h->aux) {
    e = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking);
    cudaEvent_t* evs[6] = {&h->ev_fwd, &h->ev_aux_end, &h->ev_rec[0], &h->ev_rec[1], &h->ev_adj[0], &h->ev_adj[1]};
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(evs[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: stream and events");
  }
  auto ckpt = [&](int c) { return ws + L.ckpt + (size_t)c * L.state; };
  auto seg_len = [&](int c) { return H - c * K < K ? H - c * K : K; };
  // state j (0..len) of segment c and its clock slot
  auto st_at = [&](int c, int j) {
    if (j == 0) return ckpt(c);
    if (j == seg_len(c) && c + 1 < n_ck) return ckpt(c + 1);
    return ws + L.seg[c & 1] + (size_t)(j - 1) * L.state;
  };
  auto clk_at = [&](int c, int j) {
    if (j == 0) return clk + c;
    if (j == seg_len(c) && c + 1 < n_ck) return clk + c + 1;
    return clk + n_ck + (c & 1) * K + (j - 1);
  };
  // The forward pass keeps only the checkpoints and the last segment: the
  // inner states of the other segments alternate between two slots of the
  // segment buffer the last segment does not use (they stay in L2; the
  // backward pass recomputes them).
  const int last = n_ck - 1;
  auto fw_at = [&](int c, int j) {
    if (c == last || j == 0 || j == seg_len(c)) return st_at(c, j);
    return ws + L.seg[(last + 1) & 1] + (size_t)((j - 1) & 1) * L.state;
  };
  auto fw_clk = [&](int c, int j) {
    if (c == last || j == 0 || j == seg_len(c)) return clk_at(c, j);
    return clk + n_ck + ((last + 1) & 1) * K + ((j - 1) & 1);
  };
  auto step = [&](int c, int j, cudaStream_t st, bool forward_pass) {
    gpflbm::StepIO io;
    unsigned char* in = forward_pass ? fw_at(c, j) : st_at(c, j);
    unsigned char* out = forward_pass ? fw_at(c, j + 1) : st_at(c, j + 1);
    io.phi_in = in;
    io.mu_in = in + pl;
    io.f_in = in + 2 * pl;
    io.phi_out = out;
    io.mu_out = out + pl;
    io.f_out = out + 2 * pl;
    io.clock_in = forward_pass ? fw_clk(c, j) : clk_at(c, j);
    io.clock_out = forward_pass ? fw_clk(c, j + 1) : clk_at(c, j + 1);
    io.flags_in = nullptr;  // 2D: no liquid-tile flags
    io.flags_out = nullptr;
    return stepper(h)->step(P, io, st);
  };
  // copies of one stored state: handle -> slot, or slot -> handle
  auto copy_state = [&](unsigned char* slot, double* slot_clk, bool to_slot) {
    void* hp[4] = {at(h, h->lay.phi[h->cur]), at(h, h->lay.mu[h->cur]), at(h, h->lay.f[h->cur]),
                   reinterpret_cast<double*>(at(h, h->lay.clock)) + h->cur};
    void* sp[4] = {slot, slot + pl, slot + 2 * pl, slot_clk};
    const size_t n[4] = {pl, pl, 9 * pl, sizeof(double)};
    cudaError_t r = cudaSuccess;
    for (int i = 0; i < 4 && r == cudaSuccess; ++i)
      r = cudaMemcpyAsync(to_slot ? sp[i] : hp[i], to_slot ? hp[i] : sp[i], n[i], cudaMemcpyDeviceToDevice, s);
    return r;
  };

  // forward pass: checkpoints, and the last segment kept whole
  e = copy_state(ckpt(0), clk, true);
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: checkpoint copy");
  for (int c = 0; c < n_ck; ++c)
    for (int j = 0; j < seg_len(c); ++j) {
      e = step(c, j, s, true);
      if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: forward step");
    }
  e = copy_state(st_at(last, seg_len(last)), clk_at(last, seg_len(last)), false);
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: final state");
  h->t += H;

  // objective of the final state and the adjoint state it seeds
  unsigned char* lam[2] = {ws + L.lam[0], ws + L.lam[1]};
  double* gacc = reinterpret_cast<double*>(ws + L.gacc);
  double* partial = reinterpret_cast<double*>(ws + L.partial);
  double* tip = reinterpret_cast<double*>(ws + L.tip);
  const long long want = (h->cells + gpflbm::kRedThreads - 1) / gpflbm::kRedThreads;
  const int blocks = (int)(want < gpflbm::kRedMaxBlocks ? want : gpflbm::kRedMaxBlocks);
  const void* s_fin = st_at(last, seg_len(last));
  const bool on_device = (dst_is_device & GPFLBM_ON_DEVICE) != 0;
  const size_t exch = (size_t)h->cells * h->ops->real_size;  // one exchange plane
  if (obj) {
    e = A->frac(P, s_fin, partial, blocks, s);
    if (e == cudaSuccess) e = A->init(P, s_fin, obj->w_frac, lam[0], lam[0] + pl, lam[0] + 2 * pl, gacc, s);
    if (e == cudaSuccess) e = A->tip(P, s_fin, obj->x0, obj->y0, obj->kappa, obj->w_tip, lam[0], tip, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: objective");
  } else {
    // lambda^{t0+H} = seed, plane by plane (host planes through the stage area)
    e = cudaMemsetAsync(lam[0], 0, L.state, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gacc, 0, 3 * (size_t)h->plane * sizeof(double), s);
    for (int k = 0; k < 11 && e == cudaSuccess; ++k) {
      const unsigned char* src = static_cast<const unsigned char*>(seed) + (size_t)k * exch;
      if (!on_device) {
        e = cudaMemcpyAsync(at(h, h->lay.stage), src, exch, cudaMemcpyHostToDevice, s);
        src = static_cast<const unsigned char*>(at(h, h->lay.stage));
      }
      if (e == cudaSuccess) e = A->import_plane(P, src, lam[0] + (size_t)k * pl, s);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "vjp: seed");
  }

  // backward: segment c's adjoint steps on `s` while segment c-1 is
  // recomputed on the auxiliary stream
  e = cudaEventRecord(h->ev_fwd, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux, h->ev_fwd, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: stream order");
  int cur = 0;
  for (int c = last; c >= 0; --c) {
    if (c >= 1) {
      // segment c-1 reuses the slots segment c+1 was read from
      if (c + 1 <= last) e = cudaStreamWaitEvent(h->aux, h->ev_adj[(c + 1) & 1], 0);
      for (int j = 0; j + 1 < seg_len(c - 1) && e == cudaSuccess; ++j) e = step(c - 1, j, h->aux, false);
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_rec[(c - 1) & 1], h->aux);
      if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: recompute");
    }
    if (c < last) {
      e = cudaStreamWaitEvent(s, h->ev_rec[c & 1], 0);
      if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: stream order");
    }
    for (int j = seg_len(c) - 1; j >= 0; --j) {
      gpflbm::AdjStepIO a;
      unsigned char* s0 = st_at(c, j);
      unsigned char* s1 = st_at(c, j + 1);
      a.s0 = s0;
      a.mu0 = s0 + pl;
      a.d0 = s0 + 2 * pl;
      a.s1 = s1;
      a.mu1 = s1 + pl;
      a.ls1 = lam[cur];
      a.lmu1 = lam[cur] + pl;
      a.ld1 = lam[cur] + 2 * pl;
      a.ls0 = lam[1 - cur];
      a.lmu0 = lam[1 - cur] + pl;
      a.ld0 = lam[1 - cur] + 2 * pl;
      a.gacc = gacc;
      a.clock = clk_at(c, j);
      e = A->step(P, a, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: step");
      cur = 1 - cur;
    }
    e = cudaEventRecord(h->ev_adj[c & 1], s);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: stream order");
  }
  e = cudaEventRecord(h->ev_aux_end, h->aux);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_aux_end, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: stream order");

  // outputs
  if (grad) {
    for (int k = 0; k < 11 && e == cudaSuccess; ++k) {
      unsigned char* dst = static_cast<unsigned char*>(grad) + (size_t)k * exch;
      e = A->export_plane(P, lam[cur] + (size_t)k * pl, on_device ? dst : at(h, h->lay.stage), s);
      if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(dst, at(h, h->lay.stage), exch, cudaMemcpyDeviceToHost, s);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "vjp: gradient");
  }
  if (dmu0) {
    void* target = on_device ? dmu0 : at(h, h->lay.stage);
    e = A->export_plane(P, lam[cur] + pl, target, s);
    if (e == cudaSuccess && !on_device)
      e = cudaMemcpyAsync(dmu0, target, (size_t)h->cells * h->ops->real_size, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: dmu0");
  }
  for (int j = 0; j < 3 && e == cudaSuccess; ++j)
    e = A->sum(P, gacc + (size_t)j * h->plane, partial + (size_t)(j + 1) * gpflbm::kRedMaxBlocks, blocks, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: parameter sums");
  std::vector<double> host(4 * (size_t)gpflbm::kRedMaxBlocks + 1);
  e = cudaMemcpyAsync(host.data(), partial, 4 * (size_t)gpflbm::kRedMaxBlocks * sizeof(double),
                      cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&host[4 * (size_t)gpflbm::kRedMaxBlocks], tip, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: results");
  double sums[4];
  for (int j = 0; j < 4; ++j) {
    double t = 0.0;
    for (int b = 0; b < blocks; ++b) t += host[(size_t)j * gpflbm::kRedMaxBlocks + b];
    sums[j] = t;
  }
  const double tip_v = host[4 * (size_t)gpflbm::kRedMaxBlocks];
  if (J && obj) *J = obj->w_frac * (sums[0] / (double)h->cells) + obj->w_tip * tip_v / (double)h->grid.nx;
  if (dparams)
    for (int j = 0; j < 3; ++j) dparams[j] = sums[j + 1];
  return GPFLBM_OK;
}

}  // namespace

extern "C" {

gpflbm_status gpflbm_adjoint_workspace_bytes(gpflbm_t h, int horizon, int ckpt_every, size_t* bytes) {
  if (!h || !bytes) return GPFLBM_ERR_ARG;
  gpflbm_status st = adj_check(h, horizon, ckpt_every);
  if (st != GPFLBM_OK) return st;
  *bytes = adj_layout(h, horizon, ckpt_every).total;
  return GPFLBM_OK;
}

gpflbm_status gpflbm_adjoint(gpflbm_t h, const gpflbm_objective* obj, int horizon, int ckpt_every,
                             void* workspace, size_t workspace_bytes, double* J, double* dparams,
                             void* dmu0, int dst_is_device, void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  gpflbm_status st = adj_check(h, horizon, ckpt_every);
  if (st != GPFLBM_OK) return st;
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, "adjoint: no state loaded");
  if (dst_is_device & ~(GPFLBM_ON_DEVICE | GPFLBM_ASYNC))
    return fail(h, GPFLBM_ERR_ARG, "adjoint: unknown flag");
  ++h->mut;
  if (!obj || obj->solid != 1 || obj->x0 < 0 || obj->x0 >= h->grid.nx || obj->y0 < 0 ||
      obj->y0 >= h->grid.ny || !std::isfinite(obj->kappa) || !std::isfinite(obj->w_frac) ||
      !std::isfinite(obj->w_tip))
    return fail(h, GPFLBM_ERR_ARG, "adjoint: invalid objective (solid must be 1, (x0, y0) inside)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const AdjLayout L = adj_layout(h, horizon, ckpt_every);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  bool own = false;
  if (ws) {
    if (workspace_bytes < L.total) return fail(h, GPFLBM_ERR_OOM, "adjoint: workspace too small");
    if (reinterpret_cast<uintptr_t>(ws) % kAlign != 0)
      return fail(h, GPFLBM_ERR_ARG, "adjoint: workspace not 256-byte aligned");
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, L.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, GPFLBM_ERR_OOM, "adjoint: cudaMalloc of the workspace failed");
    }
    ws = static_cast<unsigned char*>(p);
    own = true;
  }
  st = adjoint_run(h, obj, horizon, L, ws, J, dparams, dmu0, dst_is_device, s);
  if (own) {
    cudaStreamSynchronize(s);  // nothing may still use the block
    cudaFree(ws);
  }
  return st;
}

gpflbm_status gpflbm_vjp(gpflbm_t h, int horizon, int ckpt_every, void* workspace, size_t workspace_bytes,
                         const void* seed, void* grad, double* dparams, int flags, void* stream) {
  if (!h) return GPFLBM_ERR_ARG;
  gpflbm_status st = adj_check(h, horizon, ckpt_every);
  if (st != GPFLBM_OK) return st;
  if (!h->has_state) return fail(h, GPFLBM_ERR_STATE, "vjp: no state loaded");
  if (flags & ~(GPFLBM_ON_DEVICE | GPFLBM_ASYNC)) return fail(h, GPFLBM_ERR_ARG, "vjp: unknown flag");
  if (!seed) return fail(h, GPFLBM_ERR_ARG, "vjp: seed is NULL");
  ++h->mut;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const AdjLayout L = adj_layout(h, horizon, ckpt_every);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  bool own = false;
  if (ws) {
    if (workspace_bytes < L.total) return fail(h, GPFLBM_ERR_OOM, "vjp: workspace too small");
    if (reinterpret_cast<uintptr_t>(ws) % kAlign != 0)
      return fail(h, GPFLBM_ERR_ARG, "vjp: workspace not 256-byte aligned");
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, L.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, GPFLBM_ERR_OOM, "vjp: cudaMalloc of the workspace failed");
    }
    ws = static_cast<unsigned char*>(p);
    own = true;
  }
  st = adjoint_run(h, nullptr, horizon, L, ws, nullptr, dparams, nullptr, flags, s, seed, grad);
  if (own) {
    cudaStreamSynchronize(s);
    cudaFree(ws);
  }
  return st;
}

}  // extern "C"

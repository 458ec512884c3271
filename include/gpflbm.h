/*
 * gpflbm.h -- C ABI of the GB300 (sm_103a) library for the coupled
 * Grand-Potential phase-field / lattice-Boltzmann time step.
 *
 * One step advances the state S^n = {f_k (Q planes), phi_a (N planes),
 * mu_i (K-1 planes)} to S^{n+1} in the order of the paper's Algorithm 1:
 *   1. phase-field update, Eq. PhfGrand with the obstacle potential of
 *      Eq. Wpot, a Lagrange multiplier over the locally present phases and
 *      a Euclidean projection onto the Gibbs simplex (Sec. 2.1);
 *   2. chemical-potential update, Eq. conc, in flux form: diffusion,
 *      antitrapping, the c_a dh_a/dt source and advection by the lattice
 *      Boltzmann velocity of step n (Sec. 2.1, Algorithm 1);
 *   3. BGK collision with the second-order equilibrium (Eq. f^eq) and the
 *      discrete force (Eq. discreteForce) made of the drag G_D and the
 *      buoyancy G_B (Sec. 2.2), then streaming (Eq. LBMEq_1) with halfway
 *      bounce-back on wall axes; density and momentum from Eq. rhovel with
 *      the force-corrected velocity U = (m + F_B/2) / (rho (1 + kappa/2)).
 *
 * Conventions for every call:
 *  - Fields are structure-of-arrays planes, x fastest:
 *    index = x + nx * (y + ny * z); nz == 1 for 2D.  The vertical axis
 *    (gravity along -v) is y in 2D and z in 3D.
 *  - Element type of exchanged fields: double for GPFLBM_FP64, float for
 *    every other precision.  Populations are always exchanged as the full
 *    f_k (the library stores f_k - w_k internally).
 *  - D2Q9 numbering is the paper's lattice figure: 0 rest, 1 (+x), 2 (+y),
 *    3 (-x), 4 (-y), 5 (+x+y), 6 (-x+y), 7 (-x-y), 8 (+x-y).
 *    D3Q19 numbering: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (+1,+1,0),
 *    (-1,-1,0), (+1,-1,0), (-1,+1,0), (+1,0,+1), (-1,0,-1), (+1,0,-1),
 *    (-1,0,+1), (0,+1,+1), (0,-1,-1), (0,+1,-1), (0,-1,+1).
 *    D3Q27 (the paper's 3D set; weights 8/27, 2/27, 1/54, 1/216 by class):
 *    the D3Q19 directions, then 19..26 = (+1,+1,+1), (-1,-1,-1), (+1,+1,-1),
 *    (-1,-1,+1), (+1,-1,+1), (-1,+1,-1), (-1,+1,+1), (+1,-1,-1).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered and asynchronous unless stated otherwise.
 *  - Every call returns a gpflbm_status; nothing aborts.  After a failure
 *    gpflbm_last_error(h) describes it.  A handle is not thread-safe.
 */
#ifndef GPFLBM_H
#define GPFLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpflbm_s* gpflbm_t;

typedef enum {
  GPFLBM_OK = 0,
  GPFLBM_ERR_ARG = -1,         /* invalid argument (pointer, size, enum, range) */
  GPFLBM_ERR_OOM = -2,         /* workspace too small or device allocation failed */
  GPFLBM_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  GPFLBM_ERR_NONFINITE = -4,   /* NaN or Inf found in the state by gpflbm_invariants */
  /* -5 is not used: no kernel of the library waits on another agent */
  GPFLBM_ERR_STATE = -6,       /* call out of order (e.g. step before set_state) */
  GPFLBM_ERR_UNSUPPORTED = -7  /* valid but not built: phase/solute count, lattice */
} gpflbm_status;

enum { GPFLBM_PERIODIC = 0, GPFLBM_WALL = 1 };
enum { GPFLBM_D2Q9 = 9, GPFLBM_D3Q19 = 19, GPFLBM_D3Q27 = 27 };
enum {
  GPFLBM_FP64 = 0,           /* FP64 arithmetic and storage */
  GPFLBM_FP32 = 1,           /* FP32 arithmetic and storage */
  GPFLBM_FP32_F16STORE = 2,  /* FP32 arithmetic, f_k - w_k stored as FP16 times 2^10 */
  GPFLBM_FP32_BF16STORE = 3  /* FP32 arithmetic, f_k - w_k stored as BF16 */
};
enum {
  GPFLBM_FIELD_PHI = 1,  /* N planes, liquid (phase 0) first */
  GPFLBM_FIELD_MU = 2,   /* K-1 planes */
  GPFLBM_FIELD_C = 4,    /* K-1 planes: c_i = sum_a h_a(phi) c_a,i(mu) */
  GPFLBM_FIELD_F = 8,    /* Q planes, full populations f_k */
  GPFLBM_FIELD_RHO = 16, /* 1 plane: sum_k f_k */
  GPFLBM_FIELD_U = 32    /* d planes: force-corrected velocity of the current state (with drag
                            and buoyancy; the shrinkage force needs the next phase field and is
                            not included) */
};

#define GPFLBM_MAX_PHASES 4
#define GPFLBM_MAX_SOLUTES 2

/* Grid and storage.  bc[a]: GPFLBM_PERIODIC or GPFLBM_WALL per axis
 * (WALL = zero-flux for phi and mu, halfway bounce-back for f).
 * wall_rows[a]: static obstacle rows at both ends of axis a: phi and mu are
 * frozen there, no solute crosses their faces, and the flow sees them as
 * solid (drag with phi_l = 0, no buoyancy). */
typedef struct {
  int nx, ny, nz;    /* cells per axis; nz == 1 selects 2D */
  int lattice;       /* GPFLBM_D2Q9 (2D); GPFLBM_D3Q19 or GPFLBM_D3Q27 (3D; D3Q27 with
                        FP64 or FP32 precision only, else GPFLBM_ERR_UNSUPPORTED) */
  int bc[3];
  int wall_rows[3];
  int precision;     /* GPFLBM_FP64 ... GPFLBM_FP32_BF16STORE */
} gpflbm_grid;

/* Material and model parameters, lattice units (dx = dt = 1).  Phase 0 is
 * the liquid.  Entries beyond n_phases / n_components are ignored. */
typedef struct {
  double tau_f;                    /* BGK relaxation time, nu = (tau_f - 1/2) / 3 */
  double tau_phi;                  /* tau of Eq. PhfGrand (interface mobility = 1/tau_phi) */
  double eps;                      /* interface width parameter epsilon, cells */
  double gamma[4][4];              /* interface energy per pair (symmetric, zero diagonal) */
  double delta[4][4];              /* cubic anisotropy strength per pair (0 = isotropic) */
  double A[4];                     /* parabolic free energy f_a(c) = A_a |c - ceq_a|^2 */
  double ceq[4][2];                /* equilibrium composition per phase and solute */
  double S[4];                     /* psi_a gains S_a (T - T_E); S_0 = 0 for the liquid */
  double D_liq;                    /* liquid diffusivity; mobility M = D_liq phi_l / (2 A_0) */
  double a_at;                     /* antitrapping coefficient (0 = off) */
  double h_drag, W0;               /* drag G_D = -rho kappa U, kappa = 2 nu h (1-phi_l)^2 / W0^2 */
  double gbeta_c[2], c_ref[2];     /* solutal buoyancy g beta_i (c_l,i - c_ref,i), upward */
  double gbeta_T, T_ref;           /* thermal buoyancy g beta_T (T - T_ref), upward */
  double T_E, undercool, G, V, v0; /* T(v, t) = T_E - undercool + G (v - v0 - V t) */
  double q_floor;                  /* |q|^2 at or below which the anisotropy is dropped */
  double eta_rho[4];               /* shrinkage (rho_a - rho_0) / rho_0 per phase (Eq. shrinkage):
                                      G_S = sum_a eta_a (phi_a^{n+1} - phi_a^n) grad phi_a / |grad phi_a|
                                      joins the buoyancy in U and F; all 0 = no shrinkage */
  double tilt[4][4];               /* crystal axes of pair (a, b) turned by this angle (radians,
                                      counter-clockwise about z; symmetric, finite): the
                                      anisotropy of Eq. PhfGrand is evaluated on
                                      q' = (c q_x + s q_y, -s q_x + c q_y, q_z), c = cos, s = sin,
                                      so the fastest growth of a delta > 0 crystal points at the
                                      angle; the seed misorientation theta of the paper's
                                      dendrite cases.  All 0 = axis-aligned crystals */
  double dceq_dT[4][2];            /* temperature dependence of the equilibrium compositions:
                                      ceq_a,i(T) = ceq[a][i] + dceq_dT[a][i] (T - T_E), in c_a(mu, T),
                                      psi_a and every composition; Eq. conc gains
                                      -(dT/dt) sum_a dceq_dT[a][i] h_a (dT/dt = -G V, h at n+1).
                                      All 0 = ceq independent of T */
} gpflbm_params;

/* Device bytes the library needs for a problem (state ping-pong buffers,
 * reduction partials, step counter), for a caller that provides the memory.
 * Returns GPFLBM_ERR_ARG / GPFLBM_ERR_UNSUPPORTED for an invalid or unbuilt
 * configuration.  Does not touch the GPU. */
gpflbm_status gpflbm_workspace_bytes(const gpflbm_grid* grid, int n_phases, int n_components,
                                     size_t* bytes);

/* Create a simulation handle.  n_phases = N (2..4, phase 0 liquid),
 * n_components = K-1 independent solutes (1..2).  `workspace` is device
 * memory of at least gpflbm_workspace_bytes() bytes, 256-byte aligned, owned
 * by the caller and kept alive (and untouched) until gpflbm_destroy; pass
 * NULL to let the library allocate (and later free) it with cudaMalloc.
 * The state is undefined until gpflbm_set_state.  On failure *out is NULL. */
gpflbm_status gpflbm_create(const gpflbm_grid* grid, int n_phases, int n_components,
                            const gpflbm_params* params, void* workspace, size_t workspace_bytes,
                            gpflbm_t* out);

/* Slab decomposition of a 3D grid along the vertical axis (the paper runs
 * its solver as a domain decomposition over CPU processes, its Appendix A;
 * here one slab per GPU).  A slab handle owns the planes
 * v_begin .. v_begin + v_count - 1 (z) of `grid` and keeps two halo planes
 * on each side in its buffers.  Before every step it needs, from each
 * neighbouring slab, phi of the two planes next to it and mu and the
 * populations of the nearest plane (gpflbm_halo_pack on the neighbour,
 * a transfer of the message, gpflbm_halo_unpack here); its step then gives
 * bit for bit the values the whole grid's step gives on those planes (the
 * cells of the halo plane next to a neighbour are collided here as well, and
 * only their populations that stream into this slab are kept, so nothing
 * crosses after the step).  The vertical axis must have walls
 * (bc[2] = GPFLBM_WALL, wall_rows[2] = 0): the slabs at its ends mirror
 * their own planes there.  Fields, set_state, get_fields, the invariants
 * (each slab's own cells: the caller sums them) and the step counter act on
 * the owned planes as a grid of nx x ny x v_count cells.  gpflbm_step takes
 * n_steps <= 1 on a slab and GPFLBM_ERR_STATE unless every side with a
 * neighbour was unpacked since the last step or set_state.  Not supported on
 * a slab: shrinkage, gpflbm_shift_frame, the adjoint.  GPFLBM_ERR_ARG
 * unless 0 <= v_begin, v_count >= 2 and v_begin + v_count <= nz;
 * GPFLBM_ERR_UNSUPPORTED for a 2D grid or another vertical boundary.
 * Workspace as in gpflbm_create, sized by gpflbm_slab_workspace_bytes. */
gpflbm_status gpflbm_slab_workspace_bytes(const gpflbm_grid* grid, int v_begin, int v_count, int n_phases,
                                          int n_components, size_t* bytes);
gpflbm_status gpflbm_create_slab(const gpflbm_grid* grid, int v_begin, int v_count, int n_phases,
                                 int n_components, const gpflbm_params* params, void* workspace,
                                 size_t workspace_bytes, gpflbm_t* out);

/* Bytes of one halo message of a slab (the same for both sides):
 * (2 * stored phi components + K-1) planes of the arithmetic type and Q
 * planes of the population storage type, each of (nx rounded up to 8) * ny
 * elements. */
gpflbm_status gpflbm_halo_bytes(gpflbm_t h, size_t* bytes);

/* side: 0 = the neighbour below (smaller z), 1 = the neighbour above.
 * gpflbm_halo_pack writes what that neighbour needs from this slab's current
 * state into msg (device memory of gpflbm_halo_bytes, 16-byte aligned,
 * owned by the caller); gpflbm_halo_unpack writes a message packed by that
 * neighbour (its opposite side) into this slab's halo planes.  Both are
 * asynchronous on `stream`; the caller orders the transfer between them
 * (a copy on one GPU, ncclSend/ncclRecv or a peer copy between GPUs).
 * GPFLBM_ERR_ARG for a side without a neighbour (a wall), a NULL or
 * misaligned message; GPFLBM_ERR_UNSUPPORTED if h is not a slab;
 * GPFLBM_ERR_STATE before set_state. */
gpflbm_status gpflbm_halo_pack(gpflbm_t h, int side, void* msg, void* stream);
gpflbm_status gpflbm_halo_unpack(gpflbm_t h, int side, const void* msg, void* stream);

/* Replace the model parameters (same grid, phase and solute counts). */
gpflbm_status gpflbm_set_params(gpflbm_t h, const gpflbm_params* params);

/* Flags of the src_is_device / dst_is_device arguments of gpflbm_set_state
 * and gpflbm_get_fields (0 = host memory, returned to the caller complete).
 * GPFLBM_ON_DEVICE: the pointers are device memory.
 * GPFLBM_ASYNC: with device or pinned (page-locked or registered) host
 * buffers the call does not synchronise `stream`; as with cudaMemcpyAsync on
 * page-locked memory, the caller keeps the sources alive and unchanged, and
 * reads the destinations, only once the stream has reached that point.
 * Pageable host buffers are staged and waited for whatever the flag. */
#define GPFLBM_ON_DEVICE 1
#define GPFLBM_ASYNC 2

/* Load S^n.  phi: N planes (liquid first); mu: K-1 planes; f: Q planes of
 * full populations, or NULL for the fluid at rest (f_k = w_k).
 * src_is_device: flags as above (1 = device memory, 0 = host memory,
 * pageable or pinned).  The library copies; the caller keeps ownership.
 * Device and pinned or registered host sources (all three of them) are read
 * in place by one load kernel (over the host link for host memory);
 * pageable ones are staged through the workspace plane by plane.  Sets the
 * step counter to t0.  Host sources are read before return unless
 * GPFLBM_ASYNC is given with pinned sources.  With GPFLBM_ASYNC and device
 * or pinned sources (and a state already loaded) the load goes into the
 * handle's idle buffer on a stream of the library, after the work queued on
 * `stream` by the last call other than get_fields, get_deviations and the
 * invariants, so that it overlaps those read-only calls; `stream` then waits
 * for the load.  GPFLBM_ERR_ARG for an unknown flag bit. */
gpflbm_status gpflbm_set_state(gpflbm_t h, const void* phi, const void* mu, const void* f,
                               int src_is_device, long long t0, void* stream);

/* Advance n_steps >= 0 steps on `stream` (asynchronous).  Steps are
 * replayed from a CUDA graph captured on first use. */
gpflbm_status gpflbm_step(gpflbm_t h, int n_steps, void* stream);

/* Moving frame of the directional-solidification case (Sec. "Case 2:
 * Directional Solidification": the window follows the growth front).  Moves
 * the state `rows` cells down the vertical axis (y in 2D, z in 3D, the axis
 * of the temperature gradient G): layer v takes the values of layer
 * v + rows (phi, mu and the stored populations, copied exactly), the top
 * `rows` layers repeat the old top layer (a zero-gradient far field), and
 * params.v0 is lowered by `rows`, so that the frozen temperature
 * T = T_E - undercool + G (v - v0 - V t) stays with the material.  The step
 * counter is unchanged.  Asynchronous on `stream`, ordered after earlier
 * steps on it.  GPFLBM_ERR_ARG unless 0 <= rows < the vertical size;
 * GPFLBM_ERR_UNSUPPORTED with obstacle rows on the vertical axis
 * (wall_rows != 0 there); GPFLBM_ERR_STATE before set_state. */
gpflbm_status gpflbm_shift_frame(gpflbm_t h, int rows, void* stream);

/* One step launched directly (not from a graph) that records two caller
 * CUDA events (cudaEvent_t) on `stream`: events[0] before the step's
 * kernels and events[1] after them (gpflbm_step_launches launches, all
 * three updates fused in each), for kernel timing with
 * cudaEventElapsedTime.  Same result as gpflbm_step(h, 1, stream). */
gpflbm_status gpflbm_step_timed(gpflbm_t h, void* const* events, void* stream);

/* Copy fields of the current state out.  field_mask is an OR of
 * GPFLBM_FIELD_*; dst holds one pointer per set bit, in increasing bit
 * order, each large enough for that field's planes.  dst_is_device: flags
 * as in set_state.  Device and pinned host destinations are written by one
 * kernel launch; pageable host destinations are staged field by field.  For
 * host destinations the call synchronises `stream`, unless GPFLBM_ASYNC is
 * given and every destination is pinned.  GPFLBM_ERR_ARG for an unknown flag
 * bit. */
gpflbm_status gpflbm_get_fields(gpflbm_t h, unsigned field_mask, void* const* dst,
                                int dst_is_device, void* stream);

/* Stored population deviations f_k - w_k of the current state, as Q planes
 * of the exchange type (float or double), for checks of the storage codec.
 * dst_is_device: GPFLBM_ON_DEVICE for device memory, else host memory
 * (staged; the call synchronises `stream`; GPFLBM_ASYNC is accepted and
 * changes nothing).  GPFLBM_ERR_ARG for an unknown flag bit. */
gpflbm_status gpflbm_get_deviations(gpflbm_t h, void* dst, int dst_is_device, void* stream);

/* Global totals in FP64, by a fixed-order reduction (identical from run to
 * run): mass = sum_x sum_k (f_k - w_k) + cells, solute[i] = sum_x c_i,
 * solid_frac = (1/cells) sum_x sum_{a>0} h_a, with c_i at the state's time
 * (ceq_a,i(T) = ceq + dceq_dT (theta_t + G v), theta_t = -undercool - G v0
 * - G V t, when dceq_dT is not all 0).  Per cell, values are widened
 * to FP64 first and combined without fused multiply-add.  Order: 256-thread
 * blocks, grid G = min(ceil(cells/256), 608); thread t of block b adds the
 * cells b*256 + t + j*G*256 (j = 0, 1, ...) in turn; a warp combines by
 * xor-butterfly (offsets 16, 8, 4, 2, 1); lane 0 of warps 0..7 are then
 * added in order; the G block sums are added in order.  Synchronises
 * `stream`.  Returns GPFLBM_ERR_NONFINITE (totals still written) if any
 * cell of the state is NaN or Inf.  Any output pointer may be NULL. */
gpflbm_status gpflbm_invariants(gpflbm_t h, double* mass, double* solute, double* solid_frac,
                                void* stream);

/* The totals of gpflbm_invariants for callers that cannot allocate device
 * memory when they ask for them (device memory held by another framework's
 * caching allocator, or a monitoring hook that must not call the allocator
 * during a run).  The paper has no counterpart: this is a library facility.
 * The reduction scratch is a fixed 80 KB device array inside the library
 * (one per GPU that loads it, kept until the process exits), not the
 * handle's workspace; nothing is allocated.  Limit: grids of at most
 * 16,777,216 cells (larger ones return GPFLBM_ERR_ARG with a message).  The
 * totals are summed in blocks of up to 8192 cells, in a different order than
 * gpflbm_invariants, so they agree with it to FP64 rounding, not bit for
 * bit.  The first call on a device looks the array up (with that device
 * current) and should come before any stream capture; the address found is
 * kept for the life of the process, so it does not survive a
 * cudaDeviceReset (after one, handles and this entry point on that device
 * are not usable).  Calls share the array: calls that overlap on the GPU
 * race.  Synchronises `stream`; outputs and statuses (GPFLBM_ERR_NONFINITE,
 * GPFLBM_ERR_STATE) as for gpflbm_invariants. */
gpflbm_status gpflbm_invariants_noalloc(gpflbm_t h, double* mass, double* solute,
                                        double* solid_frac, void* stream);

/* Objective of gpflbm_adjoint, a function of the final state only:
 *   J = w_frac * (1/cells) sum_x h_1(phi(x))            (solid fraction)
 *     + w_tip * tip / nx,
 *   tip = sum_r r p_r,  p = softmax_r(kappa r phi_1(x0 + r, y0)),
 *   r = 0 .. nx-1-x0: a soft-argmax of the solid front along the +x ray
 * through (x0, y0).  z0 is ignored in 2D; `solid` must be 1. */
typedef struct {
  double w_frac, w_tip, kappa;
  int x0, y0, z0;
  int solid;
} gpflbm_objective;

/* Device bytes gpflbm_adjoint needs for `horizon` steps and checkpoints
 * every `ckpt_every` steps: ceil(horizon/ckpt_every) checkpoints and two
 * sets of ckpt_every recomputed states (11 planes each), two adjoint states
 * and 3 FP64 accumulator planes. */
gpflbm_status gpflbm_adjoint_workspace_bytes(gpflbm_t h, int horizon, int ckpt_every, size_t* bytes);

/* Reverse-mode derivative of the discrete map from the current state S^t0
 * through `horizon` = H steps to J(S^{t0+H}).  The paper defines the step
 * (the three updates above); the adjoint is the exact transpose of that
 * discrete step, with the simplex projection differentiated by its active
 * set: zero through a clamped phase value, the identity where one phase
 * fills the neighbourhood (the update is then phi^{n+1} = phi^n).
 * Checkpointing: a forward pass stores S every K = ckpt_every steps and
 * keeps the last segment whole; then, from the last segment back, K adjoint
 * steps run backwards through each segment while the segment before it is
 * recomputed from its checkpoint on a second stream (the library's own).
 * Cost: H + (ceil(H/K) - 1)(K - 1) forward steps plus H adjoint steps.
 * Supported: 2D, D2Q9, two phases, one solute, GPFLBM_FP64 or GPFLBM_FP32,
 * no shrinkage (eta_rho all 0); tilted crystal axes and temperature-dependent ceq are
 * supported.  Anything else: GPFLBM_ERR_UNSUPPORTED.
 * Outputs (each may be NULL): *J; dparams[0] = dJ/d(1/tau_phi),
 * dparams[1] = dJ/d delta_01, dparams[2] = dJ/d gbeta_c[0] (FP64,
 * accumulated per cell in FP64 and summed in a fixed order); dmu0 =
 * dJ/dmu(S^t0) as one plane in the exchange layout and type, device memory
 * when dst_is_device has GPFLBM_ON_DEVICE, else host memory (GPFLBM_ASYNC is
 * accepted and changes nothing; GPFLBM_ERR_ARG for an unknown flag bit).
 * Every contribution is gathered in a fixed
 * order, so the results are the same from run to run.
 * The handle is left at S^{t0+H}, bit for bit as after gpflbm_step(h, H).
 * workspace: device memory of gpflbm_adjoint_workspace_bytes() bytes,
 * 256-byte aligned, or NULL for a cudaMalloc'd block freed before return.
 * Synchronises `stream`. */
gpflbm_status gpflbm_adjoint(gpflbm_t h, const gpflbm_objective* obj, int horizon, int ckpt_every,
                             void* workspace, size_t workspace_bytes, double* J, double* dparams,
                             void* dmu0, int dst_is_device, void* stream);

/* Vector-Jacobian product of the discrete map from the current state S^t0
 * through `horizon` = H steps: the same reverse sweep, checkpointing and
 * configurations as gpflbm_adjoint, for the linear functional
 *   J = sum_x [ seed_s phi_1 + seed_mu mu + sum_k seed_k f_k ](S^{t0+H})
 * instead of the objective.  seed: 11 planes in the exchange layout and type
 * (phi_1, mu, f_0 .. f_8; phi_0 = 1 - phi_1 is not a free variable of the
 * two-phase state).  grad (may be NULL): the 11 planes of dJ/dS^t0 in the
 * same layout (dJ/dphi_1, dJ/dmu, dJ/df_k).  dparams (may be NULL): as in
 * gpflbm_adjoint.  flags: GPFLBM_ON_DEVICE when seed and grad are device
 * memory, else host memory (staged plane by plane); GPFLBM_ASYNC is
 * accepted and changes nothing.  Workspace as for gpflbm_adjoint.  The
 * handle is left at S^{t0+H}.  Synchronises `stream`. */
gpflbm_status gpflbm_vjp(gpflbm_t h, int horizon, int ckpt_every, void* workspace, size_t workspace_bytes,
                         const void* seed, void* grad, double* dparams, int flags, void* stream);

/* Kernel launches one step makes with the current parameters: 1 or 2.
 * In 3D the tiles whose reach is pure liquid take a lean path and the
 * others the general one (not on slabs, nor with shrinkage or obstacle
 * rows); each tile is advanced by exactly one of them.  Two phases with
 * FP32 arithmetic on D3Q19: one launch runs both paths (the general tiles
 * start first).  Otherwise the general kernel runs, then the liquid-tile
 * kernel: 2.  Every other case: 1.  Does not touch the GPU. */
gpflbm_status gpflbm_step_launches(gpflbm_t h, int* launches);

/* Step counter of the current state (the t of T(v, t)). */
gpflbm_status gpflbm_time(gpflbm_t h, long long* t);

/* Human-readable description of the last failure on h ("" if none). */
const char* gpflbm_last_error(gpflbm_t h);

/* Release the handle (and the workspace if the library allocated it).
 * Waits for the handle's own transfer stream (asynchronous loads); work the
 * caller queued on its streams is the caller's to wait for before freeing a
 * workspace it owns. */
void gpflbm_destroy(gpflbm_t h);

#ifdef __cplusplus
}
#endif

#endif /* GPFLBM_H */

// ORACLE — test infrastructure only.
//
// A plain, slow, FP64 CPU statement of one time step of the Grand-Potential
// phase-field / lattice-Boltzmann model (Sec. 2, Eq. PhfGrand, Eq. conc,
// Eq. LBMEq_1 .. Eq. rhovel, Algorithm 1 of the paper).  Only the test suite,
// the smoke check and the CPU-baseline leg of the benchmark load this file;
// the product path (the CUDA library) never does, and the two share no code:
// this file includes no header of the CUDA library and the CUDA library
// includes nothing from here.
//
// Everything is written cell by cell in the order the paper's Algorithm 1
// gives (phase field -> chemical potential -> lattice Boltzmann), with no
// blocking or fusion, so that each line can be read against an equation.
// Where the paper leaves a choice open, the reading taken is named [Rn] at
// the place it is used; the list of readings is kept with the design notes.
//
// The scalar type is a template parameter: `double` for the plain run, and
// `Dual` (value + one tangent) for exact forward-mode directional
// derivatives, which is how the oracle's gradient is obtained.  Branches
// (active set, projection, thresholds) are taken on the value part, so the
// dual run differentiates the same piecewise-smooth map the value run
// evaluates (the active-set subgradient).
//
// Pins (tests/test_oracle_pins.py): flat-interface equilibrium profile and
// compositions, textbook 5/7-point Laplacian for the isotropic two-phase
// case, 1+delta*cos(4 theta) anisotropy, interpolation sum rule, FTCS heat
// kernel for frozen liquid, Taylor-Green decay, Poiseuille between walls,
// uniform body force, lattice moment identities, exact conservation,
// quiescent melt, the thin-interface chemical-potential jump of a slowly
// moving planar front with and without the antitrapping current, a
// manufactured solution for the anisotropic face fluxes, and the closed-form
// soft-argmax of a sharp step for the objective.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
// Problem description.  Field layout everywhere: structure of arrays, one
// plane per component, x fastest: index = x + nx*(y + ny*z).
typedef struct {
  int nx, ny, nz;      // cells per axis (nz == 1 in 2D)
  int dim;             // 2 or 3
  int q;               // 9 (D2Q9), 19 (D3Q19) or 27 (D3Q27)
  int n_phases;        // N; phase 0 is the liquid
  int n_solutes;       // K-1 independent chemical potentials
  int bc[3];           // per axis: 0 periodic, 1 wall
  int wall_rows[3];    // static obstacle rows at both ends of each axis
  double tau_f;        // BGK relaxation time
  double tau_phi;      // phase-field relaxation constant tau of Eq. PhfGrand
  double eps;          // interface width parameter epsilon (cells)
  double gamma[4][4];  // interface energies gamma_ab
  double delta[4][4];  // cubic anisotropy strength per pair
  double A[4];         // parabolic free-energy curvature per phase
  double ceq[4][2];    // equilibrium composition per phase and solute
  double S[4];         // temperature coupling of psi per phase
  double D_liq;        // liquid diffusivity (lattice units)
  double a_at;         // antitrapping coefficient (0 = off)
  double h_drag, W0;   // drag constant h and interface thickness W0
  double gbeta_c[2];   // solutal buoyancy g*beta per solute
  double c_ref[2];     // reference liquid composition
  double gbeta_T;      // thermal buoyancy g*beta_T
  double T_ref;        // reference temperature for the thermal buoyancy
  double T_E;          // eutectic / equilibrium temperature
  double undercool;    // T = T_E - undercool + G (v - v0 - V t)
  double G, V, v0;
  double q_floor;      // |q|^2 at or below which the anisotropy is dropped
  double eta[4];       // shrinkage (rho_a - rho_liq) / rho_liq per phase, Eq. shrinkage
  double tilt[4][4];   // crystal axes of a pair turned by this angle about z (radians)
  double dceq_dT[4][2];  // slope of the equilibrium composition with temperature
} OracleProblem;

// Objective for the gradient checks: J = w_frac * mean_x sum_{a>0} h_a(phi)
//   + w_tip * tip / L, tip the soft-argmax of r*phi_s(r) along the +x ray
//   through (x0, y0[, z0]) with sharpness kappa.
typedef struct {
  double w_frac, w_tip, kappa;
  int x0, y0, z0;
  int solid;  // phase whose tip is tracked
} OracleObjective;
}

namespace {

const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
inline Dual exp(Dual a) {
  double e = std::exp(a.v);
  return Dual(e, e * a.d);
}
// Counting number: a double whose +, -, *, /, sqrt and exp each add one to
// a global tally (the floating-point operations of the method, counted by
// running the same templated steps on it; single-threaded).
long long g_flops = 0;
struct Cnt {
  double v;
  Cnt(double a = 0.0) : v(a) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_flops; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_flops; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_flops; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_flops; return Cnt(a.v / b.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { a = a * b; return a; }
inline Cnt sqrt(Cnt a) { ++g_flops; return Cnt(std::sqrt(a.v)); }
inline Cnt exp(Cnt a) { ++g_flops; return Cnt(std::exp(a.v)); }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double val(const Cnt& x) { return x.v; }
using std::exp;
using std::sqrt;

// ---------------------------------------------------------------- lattices
// D2Q9 in the numbering of the paper's lattice figure; D3Q19 rest, the six
// faces and the twelve edges, each direction followed by its opposite;
// D3Q27 adds the eight corners after them.
struct Lattice {
  int q;
  int c[27][3];
  double w[27];
  int opp[27];
};

Lattice make_lattice(int q) {
  Lattice L;
  L.q = q;
  if (q == 9) {
    const int c[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                         {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    for (int k = 0; k < 9; ++k) {
      L.c[k][0] = c[k][0];
      L.c[k][1] = c[k][1];
      L.c[k][2] = 0;
      L.w[k] = k == 0 ? 4.0 / 9.0 : (k < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
  } else {
    // rest, the 6 faces, the 12 edges (D3Q19), then for D3Q27 the 8
    // corners (+-1, +-1, +-1), as the classes of the paper's lattice table
    const int c[27][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                          {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                          {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                          {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
                          {1, 1, 1},  {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
                          {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
    for (int k = 0; k < q; ++k) {
      for (int a = 0; a < 3; ++a) L.c[k][a] = c[k][a];
      if (q == 19)
        L.w[k] = k == 0 ? 1.0 / 3.0 : (k < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
      else
        L.w[k] = k == 0 ? 8.0 / 27.0 : (k < 7 ? 2.0 / 27.0 : (k < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
  }
  for (int k = 0; k < q; ++k)
    for (int j = 0; j < q; ++j)
      if (L.c[j][0] == -L.c[k][0] && L.c[j][1] == -L.c[k][1] && L.c[j][2] == -L.c[k][2])
        L.opp[k] = j;
  return L;
}

// ---------------------------------------------------------------- grid helpers
struct Grid {
  const OracleProblem* p;
  int n[3];
  long cells;
  explicit Grid(const OracleProblem* pp) : p(pp) {
    n[0] = pp->nx;
    n[1] = pp->ny;
    n[2] = pp->dim == 3 ? pp->nz : 1;
    cells = (long)n[0] * n[1] * n[2];
  }
  long idx(int x, int y, int z) const { return x + (long)n[0] * (y + (long)n[1] * z); }
  void coords(long i, int* c) const {
    c[0] = (int)(i % n[0]);
    c[1] = (int)((i / n[0]) % n[1]);
    c[2] = (int)(i / ((long)n[0] * n[1]));
  }
  // Neighbour coordinate along one axis for the finite-difference fields:
  // periodic axes wrap, wall axes mirror across the boundary face so that the
  // normal difference across that face vanishes (Neumann, as the paper's
  // cases use for phi, c and mu).
  int fold(int i, int a) const {
    if (i < 0) return p->bc[a] == 1 ? -1 - i : i + n[a];
    if (i >= n[a]) return p->bc[a] == 1 ? 2 * n[a] - 1 - i : i - n[a];
    return i;
  }
  long nb(const int* c, int dx, int dy, int dz) const {
    return idx(fold(c[0] + dx, 0), fold(c[1] + dy, 1), p->dim == 3 ? fold(c[2] + dz, 2) : 0);
  }
  long nb(const int* c, const int* o) const { return nb(c, o[0], o[1], o[2]); }
  // Static obstacle rows (the "phase-field solid walls"), [R4].
  bool obstacle(const int* c) const {
    for (int a = 0; a < p->dim; ++a)
      if (p->wall_rows[a] > 0 && (c[a] < p->wall_rows[a] || c[a] >= n[a] - p->wall_rows[a]))
        return true;
    return false;
  }
  int vertical(const int* c) const { return p->dim == 3 ? c[2] : c[1]; }
};

// Differentiable parameters: interface mobility 1/tau_phi, anisotropy
// strengths and solutal buoyancy coefficients.
template <class R>
struct Coeffs {
  R inv_tau_phi;
  R delta[4][4];
  R gbeta_c[2];
};

template <class R>
Coeffs<R> plain_coeffs(const OracleProblem* p) {
  Coeffs<R> k;
  k.inv_tau_phi = R(1.0 / p->tau_phi);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) k.delta[a][b] = R(p->delta[a][b]);
  for (int i = 0; i < 2; ++i) k.gbeta_c[i] = R(p->gbeta_c[i]);
  return k;
}

// ---------------------------------------------------------------- thermodynamics
// Interpolation function h_a [R1]: h_a = phi_a^2 (3 - 2 phi_a)
//   + 2 phi_a sum_{b<g; b,g != a} phi_b phi_g.  sum_a h_a = 1 on the simplex.
template <class R>
R h_fn(const R* phi, int N, int a) {
  R s = 0.0;
  for (int b = 0; b < N; ++b)
    for (int g = b + 1; g < N; ++g)
      if (b != a && g != a) s += phi[b] * phi[g];
  return phi[a] * phi[a] * (3.0 - 2.0 * phi[a]) + 2.0 * phi[a] * s;
}

// dh_b / dphi_a, treating the N phase fields as independent variables.
template <class R>
R dh_fn(const R* phi, int N, int b, int a) {
  if (a == b) {
    R s = 0.0;
    for (int g = 0; g < N; ++g)
      for (int d = g + 1; d < N; ++d)
        if (g != b && d != b) s += phi[g] * phi[d];
    return 6.0 * phi[b] * (1.0 - phi[b]) + 2.0 * s;
  }
  R s = 0.0;
  for (int d = 0; d < N; ++d)
    if (d != a && d != b) s += phi[d];
  return 2.0 * phi[b] * s;
}

// Equilibrium composition of phase a at temperature T, linear in T:
// ceq_a(T) = ceq_a + (dceq_a/dT) (T - T_E).
double ceq_T(const OracleProblem* p, int a, int i, double T) {
  return p->ceq[a][i] + p->dceq_dT[a][i] * (T - p->T_E);
}

// Phase composition for the parabolic free energy
// f_a(c, T) = A_a |c - ceq_a(T)|^2:  c_a(mu, T) = ceq_a(T) + mu / (2 A_a)
// (Eq. conc uses dc_a/dmu = 1/(2 A_a) and (dc_a/dT)_mu = dceq_a/dT).
template <class R>
R c_phase(const OracleProblem* p, int a, int i, const R* mu, double T) {
  return ceq_T(p, a, i, T) + mu[i] / (2.0 * p->A[a]);
}

// Grand potential of phase a [R2]: psi_a = -|mu|^2/(4 A_a) - mu.ceq_a(T)
//   + S_a (T - T_E).
template <class R>
R psi_fn(const OracleProblem* p, int a, const R* mu, double T) {
  R s = 0.0;
  for (int i = 0; i < p->n_solutes; ++i)
    s += -mu[i] * mu[i] / (4.0 * p->A[a]) - mu[i] * ceq_T(p, a, i, T);
  return s + p->S[a] * (T - p->T_E);
}

// Analytic temperature field T(v, t) = T_E - undercool + G (v - v0 - V t).
double temperature(const OracleProblem* p, int v, double t) {
  return p->T_E - p->undercool + p->G * ((double)v - p->v0 - p->V * t);
}

// ---------------------------------------------------------------- gradient energy
// a(phi, grad phi) = sum_{a<b} gamma_ab A(q_ab), q_ab = phi_a grad phi_b
// - phi_b grad phi_a, A(q) = ac(q)^2 |q|^2 with the cubic anisotropy
// ac(q) = 1 - delta (3 - 4 sum_j q_j^4 / |q|^4)  (= 1 + delta cos 4 theta in
// 2D).  Returns dA/dq.  At |q|^2 <= q_floor the anisotropy is dropped
// (dA/dq = 2q) to avoid 0/0 [R10].
template <class R>
void dA_dq(const R* q, int dim, const R& delta, double q_floor, R* out) {
  R s2 = 0.0, s4 = 0.0;
  for (int j = 0; j < dim; ++j) {
    s2 += q[j] * q[j];
    s4 += q[j] * q[j] * q[j] * q[j];
  }
  if (val(s2) <= q_floor) {
    for (int j = 0; j < dim; ++j) out[j] = 2.0 * q[j];
    return;
  }
  R ac = 1.0 - delta * (3.0 - 4.0 * s4 / (s2 * s2));
  for (int j = 0; j < dim; ++j) {
    R dac = 16.0 * delta * (q[j] * q[j] * q[j] / (s2 * s2) - q[j] * s4 / (s2 * s2 * s2));
    out[j] = 2.0 * ac * ac * q[j] + 2.0 * ac * s2 * dac;
  }
}

// dA/dq of a pair whose crystal axes are turned by theta about the z axis
// (a tilted seed, the misorientation of the paper's dendrites): the cubic
// anisotropy is a function of the crystal components
// q' = (c qx + s qy, -s qx + c qy, qz), c = cos theta, s = sin theta, and
// dA/dq = R^T dA/dq' by the chain rule.
template <class R>
void dA_dq_tilted(const R* q, int dim, const R& delta, double theta, double q_floor, R* out) {
  if (theta == 0.0) {
    dA_dq(q, dim, delta, q_floor, out);
    return;
  }
  const double c = std::cos(theta), sn = std::sin(theta);
  R qr[3] = {c * q[0] + sn * q[1], -sn * q[0] + c * q[1], dim == 3 ? q[2] : R(0.0)};
  R d[3];
  dA_dq(qr, dim, delta, q_floor, d);
  out[0] = c * d[0] - sn * d[1];
  out[1] = sn * d[0] + c * d[1];
  if (dim == 3) out[2] = d[2];
}

// A(q) itself (same floor rule as dA_dq).
double A_value(const double* q, int dim, double delta, double q_floor) {
  double s2 = 0.0, s4 = 0.0;
  for (int j = 0; j < dim; ++j) {
    s2 += q[j] * q[j];
    s4 += q[j] * q[j] * q[j] * q[j];
  }
  if (s2 <= q_floor) return s2;
  double ac = 1.0 - delta * (3.0 - 4.0 * s4 / (s2 * s2));
  return ac * ac * s2;
}

// Value and gradient of one field plane on the face between cell c and
// c + e_d [R9]: face value = mean of the two cells; normal component = the
// difference across the face; each transverse component = the mean of the
// two cells' central differences.
template <class R>
void face_grad(const Grid& g, const R* plane, const int* c, int d, R* value, R* grad) {
  int ed[3] = {0, 0, 0};
  ed[d] = 1;
  long a = g.idx(c[0], c[1], c[2]);
  long b = g.nb(c, ed);
  *value = 0.5 * (plane[a] + plane[b]);
  for (int t = 0; t < g.p->dim; ++t) {
    if (t == d) {
      grad[t] = plane[b] - plane[a];
      continue;
    }
    int up[3] = {0, 0, 0}, dn[3] = {0, 0, 0}, bup[3], bdn[3];
    up[t] = 1;
    dn[t] = -1;
    for (int s = 0; s < 3; ++s) {
      bup[s] = ed[s] + up[s];
      bdn[s] = ed[s] + dn[s];
    }
    grad[t] = 0.25 * (plane[g.nb(c, up)] + plane[g.nb(c, bup)] - plane[g.nb(c, dn)] -
                      plane[g.nb(c, bdn)]);
  }
}

// Central-difference gradient of a plane at cell c.
template <class R>
void centre_grad(const Grid& g, const R* plane, const int* c, R* grad) {
  for (int t = 0; t < g.p->dim; ++t) {
    int up[3] = {0, 0, 0}, dn[3] = {0, 0, 0};
    up[t] = 1;
    dn[t] = -1;
    grad[t] = 0.5 * (plane[g.nb(c, up)] - plane[g.nb(c, dn)]);
  }
}

// Euclidean projection of u (length m) onto the simplex {sum = 1, u >= 0}
// by the sort-and-threshold method (Held, Wolfe & Crowder 1974; Duchi et
// al. 2008) [R11].
template <class R>
void project_simplex(R* u, int m) {
  R s[4];
  for (int j = 0; j < m; ++j) s[j] = u[j];
  std::sort(s, s + m, [](const R& a, const R& b) { return val(a) > val(b); });
  R run = 0.0, theta = 0.0;
  for (int j = 0; j < m; ++j) {
    run += s[j];
    R t = (run - 1.0) / (double)(j + 1);
    if (val(s[j]) - val(t) > 0.0) theta = t;
  }
  for (int j = 0; j < m; ++j) u[j] = val(u[j]) - val(theta) > 0.0 ? u[j] - theta : R(0.0);
}

// ---------------------------------------------------------------- the model
template <class R>
struct State {
  std::vector<R> phi, mu, f;  // N, K-1 and Q planes
};

template <class R>
struct Macro {
  std::vector<R> rho, u, F;  // rho; U and total force F, dim planes each
};

// Density, implicit-force velocity and total force at every cell from S^n
// [R5]-[R8]:  rho = sum f, m = sum c f, kappa = 2 nu h (1 - phil~)^2 / W0^2,
// F_B = rho phil~ [sum_i gbeta_i (c_l,i(mu) - c_ref,i) + gbeta_T (T - T_ref)]
// along +v, the shrinkage force of Eq. shrinkage [R26]
// F_S = sum_a eta_a (phi_a^{n+1} - phi_a^n) grad phi_a^n / |grad phi_a^n|
// (central gradient; zero where |grad|^2 <= 1e-12; absent without phi_new),
// U = (m + (F_B + F_S)/2) / (rho (1 + kappa/2)), F = F_B + F_S - rho kappa U.
template <class R>
void macroscopic(const Grid& g, const Lattice& L, const Coeffs<R>& k, const State<R>& s,
                 const std::vector<R>* phi_new, double t, Macro<R>& m) {
  const OracleProblem* p = g.p;
  const int D = p->dim, N = p->n_phases, NC = p->n_solutes;
  const long cells = g.cells;
  m.rho.assign(cells, R(0.0));
  m.u.assign(cells * D, R(0.0));
  m.F.assign(cells * D, R(0.0));
  const double nu = (p->tau_f - 0.5) / 3.0;
  const int vax = D - 1;
#pragma omp parallel for schedule(static)
  for (long x = 0; x < cells; ++x) {
    int c[3];
    g.coords(x, c);
    R rho = 0.0, mom[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < L.q; ++q) {
      R fq = s.f[q * cells + x];
      rho += fq;
      for (int a = 0; a < D; ++a) mom[a] += (double)L.c[q][a] * fq;
    }
    R phil = s.phi[0 * cells + x];
    if (g.obstacle(c)) phil = 0.0;  // obstacle rows are solid for the flow
    R kappa = 2.0 * nu * p->h_drag * (1.0 - phil) * (1.0 - phil) / (p->W0 * p->W0);
    R mu[2];
    for (int i = 0; i < NC; ++i) mu[i] = s.mu[i * cells + x];
    const double T = temperature(p, g.vertical(c), t);
    R drive = p->gbeta_T * (T - p->T_ref);
    for (int i = 0; i < NC; ++i) drive += k.gbeta_c[i] * (c_phase(p, 0, i, mu, T) - p->c_ref[i]);
    R FB = rho * phil * drive;
    R FS[3] = {R(0.0), R(0.0), R(0.0)};
    if (phi_new) {
      for (int al = 0; al < N; ++al) {
        if (p->eta[al] == 0.0) continue;
        R gr[3];
        centre_grad(g, &s.phi[al * cells], c, gr);
        R g2 = 0.0;
        for (int a = 0; a < D; ++a) g2 += gr[a] * gr[a];
        if (val(g2) <= 1e-12) continue;
        const R rate = (*phi_new)[al * cells + x] - s.phi[al * cells + x];
        const R inv = 1.0 / sqrt(g2);
        for (int a = 0; a < D; ++a) FS[a] += p->eta[al] * rate * gr[a] * inv;
      }
    }
    m.rho[x] = rho;
    for (int a = 0; a < D; ++a) {
      R num = mom[a] + 0.5 * ((a == vax ? FB : R(0.0)) + FS[a]);
      R u = num / (rho * (1.0 + 0.5 * kappa));
      m.u[a * cells + x] = u;
      m.F[a * cells + x] = (a == vax ? FB : R(0.0)) + FS[a] - rho * kappa * u;
    }
    (void)N;
  }
}

// Step 1 of Algorithm 1: phase-field update (Eq. PhfGrand with Eq. Wpot),
// explicit Euler, Lagrange multiplier over the locally active phases and
// projection onto the Gibbs simplex [R11].
template <class R>
void phase_field_update(const Grid& g, const Coeffs<R>& k, const State<R>& s, double t,
                        std::vector<R>& phi_new) {
  const OracleProblem* p = g.p;
  const int D = p->dim, N = p->n_phases, NC = p->n_solutes;
  const long cells = g.cells;
  const double eps = p->eps;

  // d-th component of da/d(grad phi_a) on the face x + e_d/2, for every
  // cell, axis and phase: -sum_{b != a} gamma_ab phi_b dA/dq(q_ab).
  std::vector<R> flux((long)D * N * cells, R(0.0));
#pragma omp parallel for schedule(static)
  for (long x = 0; x < cells; ++x) {
    int c[3];
    g.coords(x, c);
    for (int d = 0; d < D; ++d) {
      if (p->bc[d] == 1 && c[d] == g.n[d] - 1) continue;  // no flux through a wall
      R pf[4], gr[4][3];
      for (int a = 0; a < N; ++a) face_grad(g, &s.phi[a * cells], c, d, &pf[a], gr[a]);
      for (int a = 0; a < N; ++a) {
        R acc = 0.0;
        for (int b = 0; b < N; ++b) {
          if (b == a) continue;
          R qv[3], dA[3];
          for (int j = 0; j < D; ++j) qv[j] = pf[a] * gr[b][j] - pf[b] * gr[a][j];
          dA_dq_tilted(qv, D, k.delta[a][b], p->tilt[a][b], p->q_floor, dA);
          acc -= p->gamma[a][b] * pf[b] * dA[d];
        }
        flux[((long)d * N + a) * cells + x] = acc;
      }
    }
  }

#pragma omp parallel for schedule(static)
  for (long x = 0; x < cells; ++x) {
    int c[3];
    g.coords(x, c);
    R ph[4];
    for (int a = 0; a < N; ++a) ph[a] = s.phi[a * cells + x];
    if (g.obstacle(c)) {
      for (int a = 0; a < N; ++a) phi_new[a * cells + x] = ph[a];
      continue;
    }
    // divergence of the face fluxes
    R div[4];
    for (int a = 0; a < N; ++a) {
      div[a] = 0.0;
      for (int d = 0; d < D; ++d) {
        int dn[3] = {0, 0, 0};
        dn[d] = -1;
        R lower = 0.0;
        bool wall_face = p->bc[d] == 1 && c[d] == 0;
        if (!wall_face) lower = flux[((long)d * N + a) * cells + g.nb(c, dn)];
        div[a] += flux[((long)d * N + a) * cells + x] - lower;
      }
    }
    // da/dphi_a = sum_{b != a} gamma_ab dA/dq(q_ab) . grad phi_b at the centre
    R gc[4][3];
    for (int a = 0; a < N; ++a) centre_grad(g, &s.phi[a * cells], c, gc[a]);
    R dadphi[4];
    for (int a = 0; a < N; ++a) {
      dadphi[a] = 0.0;
      for (int b = 0; b < N; ++b) {
        if (b == a) continue;
        R qv[3], dA[3];
        for (int j = 0; j < D; ++j) qv[j] = ph[a] * gc[b][j] - ph[b] * gc[a][j];
        dA_dq_tilted(qv, D, k.delta[a][b], p->tilt[a][b], p->q_floor, dA);
        for (int j = 0; j < D; ++j) dadphi[a] += p->gamma[a][b] * dA[j] * gc[b][j];
      }
    }
    R mu[2];
    for (int i = 0; i < NC; ++i) mu[i] = s.mu[i * cells + x];
    double T = temperature(p, g.vertical(c), t);
    R psi[4];
    for (int b = 0; b < N; ++b) psi[b] = psi_fn(p, b, mu, T);
    // unconstrained rates g_a of Eq. PhfGrand (without Lambda)
    R rate[4];
    for (int a = 0; a < N; ++a) {
      R obst = 0.0;
      for (int b = 0; b < N; ++b)
        if (b != a) obst += p->gamma[a][b] * ph[b];
      R drive = 0.0;
      for (int b = 0; b < N; ++b) drive += psi[b] * dh_fn(ph, N, b, a);
      rate[a] = eps * (div[a] - dadphi[a]) - 16.0 / (kPi * kPi * eps) * obst - drive;
    }
    // active set: phases present anywhere in the 3^d neighbourhood
    bool active[4] = {false, false, false, false};
    int zr = D == 3 ? 1 : 0;
    for (int dz = -zr; dz <= zr; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          long y = g.nb(c, dx, dy, dz);
          for (int a = 0; a < N; ++a)
            if (val(s.phi[a * cells + y]) > 0.0) active[a] = true;
        }
    int na = 0;
    R lam = 0.0;
    for (int a = 0; a < N; ++a)
      if (active[a]) {
        lam += rate[a];
        ++na;
      }
    lam = lam / (double)na;
    // explicit Euler with dt = 1 and projection of the active phases
    R u[4];
    int ia[4], m = 0;
    for (int a = 0; a < N; ++a)
      if (active[a]) {
        u[m] = ph[a] + k.inv_tau_phi * (rate[a] - lam) / eps;
        ia[m++] = a;
      }
    project_simplex(u, m);
    for (int a = 0; a < N; ++a) phi_new[a * cells + x] = R(0.0);
    for (int j = 0; j < m; ++j) phi_new[ia[j] * cells + x] = u[j];
  }
}

// Step 2 of Algorithm 1: chemical-potential update (Eq. conc) in flux form:
// diffusion M grad mu with M = D_liq phi_l / (2 A_l) at phi^{n+1} [R12],
// antitrapping [R13] -a_at eps sum_{a>0} [phi_l]_f [c_l - c_a]_f [dphi_a]_f
// n_a.e_d (weighted by the liquid on the face: it corrects solute trapping
// at solid-liquid interfaces only), advection of h_l c_l U with U^n [R14], the source
// -sum_a c_a (h_a^{n+1} - h_a^n), and the temperature term of Eq. conc
// -(T^{n+1} - T^n) sum_a (dc_a/dT)_mu h_a^{n+1}, all divided by
// chi(phi^{n+1}).  With h at n+1 the discrete solute
// sum_a h_a c_a(mu, T) changes by exactly minus the flux divergence.
template <class R>
void chemical_potential_update(const Grid& g, const State<R>& s, const std::vector<R>& phi_new,
                               const Macro<R>& m, double t, std::vector<R>& mu_new) {
  const OracleProblem* p = g.p;
  const int D = p->dim, N = p->n_phases, NC = p->n_solutes;
  const long cells = g.cells;

  // total solute flux through the face x + e_d/2, per solute
  std::vector<R> flux((long)D * NC * cells, R(0.0));
#pragma omp parallel for schedule(static)
  for (long x = 0; x < cells; ++x) {
    int c[3];
    g.coords(x, c);
    for (int d = 0; d < D; ++d) {
      if (p->bc[d] == 1 && c[d] == g.n[d] - 1) continue;
      int ed[3] = {0, 0, 0};
      ed[d] = 1;
      long y = g.nb(c, ed);
      int cy[3];
      g.coords(y, cy);
      if (g.obstacle(c) || g.obstacle(cy)) continue;
      R mua[2], mub[2];
      for (int i = 0; i < NC; ++i) {
        mua[i] = s.mu[i * cells + x];
        mub[i] = s.mu[i * cells + y];
      }
      R Ma = p->D_liq * phi_new[0 * cells + x] / (2.0 * p->A[0]);
      R Mb = p->D_liq * phi_new[0 * cells + y] / (2.0 * p->A[0]);
      R pa[4], pb[4];
      for (int a = 0; a < N; ++a) {
        pa[a] = phi_new[a * cells + x];
        pb[a] = phi_new[a * cells + y];
      }
      R hla = h_fn(pa, N, 0), hlb = h_fn(pb, N, 0);
      R ua = m.u[d * cells + x], ub = m.u[d * cells + y];
      const double Ta = temperature(p, g.vertical(c), t), Tb = temperature(p, g.vertical(cy), t);
      for (int i = 0; i < NC; ++i) {
        R J = -0.5 * (Ma + Mb) * (mub[i] - mua[i]);
        J += 0.5 * (ua * hla * c_phase(p, 0, i, mua, Ta) + ub * hlb * c_phase(p, 0, i, mub, Tb));
        if (p->a_at != 0.0) {
          R at = 0.0;
          for (int a = 1; a < N; ++a) {
            R pf, gr[3];
            face_grad(g, &s.phi[a * cells], c, d, &pf, gr);
            R g2 = 0.0;
            for (int j = 0; j < D; ++j) g2 += gr[j] * gr[j];
            if (val(g2) <= 1e-12) continue;
            R dc = 0.5 * ((c_phase(p, 0, i, mua, Ta) - c_phase(p, a, i, mua, Ta)) +
                          (c_phase(p, 0, i, mub, Tb) - c_phase(p, a, i, mub, Tb)));
            R dphi = 0.5 * ((phi_new[a * cells + x] - s.phi[a * cells + x]) +
                            (phi_new[a * cells + y] - s.phi[a * cells + y]));
            R liq = 0.5 * (s.phi[0 * cells + x] + s.phi[0 * cells + y]);
            at += liq * dc * dphi * gr[d] / sqrt(g2);
          }
          J -= p->a_at * p->eps * at;
        }
        flux[((long)d * NC + i) * cells + x] = J;
      }
    }
  }

#pragma omp parallel for schedule(static)
  for (long x = 0; x < cells; ++x) {
    int c[3];
    g.coords(x, c);
    if (g.obstacle(c)) {
      for (int i = 0; i < NC; ++i) mu_new[i * cells + x] = s.mu[i * cells + x];
      continue;
    }
    R po[4], pn[4], mu[2];
    for (int a = 0; a < N; ++a) {
      po[a] = s.phi[a * cells + x];
      pn[a] = phi_new[a * cells + x];
    }
    for (int i = 0; i < NC; ++i) mu[i] = s.mu[i * cells + x];
    R chi = 0.0;
    for (int a = 0; a < N; ++a) chi += h_fn(pn, N, a) / (2.0 * p->A[a]);
    for (int i = 0; i < NC; ++i) {
      R div = 0.0;
      for (int d = 0; d < D; ++d) {
        int dn[3] = {0, 0, 0};
        dn[d] = -1;
        R lower = 0.0;
        if (!(p->bc[d] == 1 && c[d] == 0)) lower = flux[((long)d * NC + i) * cells + g.nb(c, dn)];
        div += flux[((long)d * NC + i) * cells + x] - lower;
      }
      const double T0 = temperature(p, g.vertical(c), t), T1 = temperature(p, g.vertical(c), t + 1.0);
      R src = 0.0;
      for (int a = 0; a < N; ++a) src += c_phase(p, a, i, mu, T0) * (h_fn(pn, N, a) - h_fn(po, N, a));
      for (int a = 0; a < N; ++a) src += (T1 - T0) * p->dceq_dT[a][i] * h_fn(pn, N, a);
      mu_new[i * cells + x] = mu[i] + (-div - src) / chi;
    }
  }
}

// Step 3 of Algorithm 1: BGK collision with the second-order equilibrium
// and Guo forcing [R15] (Eq. LBMEq_1, Eq. f^eq, Eq. discreteForce), then
// pull streaming with halfway bounce-back on wall axes.
template <class R>
void lattice_boltzmann_update(const Grid& g, const Lattice& L, const State<R>& s,
                              const Macro<R>& m, std::vector<R>& f_new) {
  const OracleProblem* p = g.p;
  const int D = p->dim;
  const long cells = g.cells;
  const double tau = p->tau_f;
  std::vector<R> fstar((long)L.q * cells);
#pragma omp parallel for schedule(static)
  for (long x = 0; x < cells; ++x) {
    R rho = m.rho[x], u[3] = {0.0, 0.0, 0.0}, F[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D; ++a) {
      u[a] = m.u[a * cells + x];
      F[a] = m.F[a * cells + x];
    }
    R uu = 0.0;
    for (int a = 0; a < D; ++a) uu += u[a] * u[a];
    for (int q = 0; q < L.q; ++q) {
      R cu = 0.0;
      for (int a = 0; a < D; ++a) cu += (double)L.c[q][a] * u[a];
      R feq = L.w[q] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
      R Gq = 0.0;
      for (int a = 0; a < D; ++a)
        Gq += (3.0 * ((double)L.c[q][a] - u[a]) + 9.0 * cu * (double)L.c[q][a]) * F[a];
      Gq = (1.0 - 0.5 / tau) * L.w[q] * Gq;
      R fq = s.f[q * cells + x];
      fstar[q * cells + x] = fq - (fq - feq) / tau + Gq;
    }
  }
#pragma omp parallel for schedule(static)
  for (long x = 0; x < cells; ++x) {
    int c[3];
    g.coords(x, c);
    for (int q = 0; q < L.q; ++q) {
      int src[3];
      bool bounce = false;
      for (int a = 0; a < 3; ++a) {
        src[a] = c[a] - L.c[q][a];
        if (a < D && (src[a] < 0 || src[a] >= g.n[a])) {
          if (p->bc[a] == 1)
            bounce = true;
          else
            src[a] = (src[a] + g.n[a]) % g.n[a];
        }
      }
      if (bounce)
        f_new[q * cells + x] = fstar[L.opp[q] * cells + x];
      else
        f_new[q * cells + x] = fstar[q * cells + g.idx(src[0], src[1], D == 3 ? src[2] : 0)];
    }
  }
}

// One full step S^n -> S^{n+1} in the order of Algorithm 1 [R8].
template <class R>
void step(const Grid& g, const Lattice& L, const Coeffs<R>& k, State<R>& s, long n) {
  const long cells = g.cells;
  const double t = (double)n;
  std::vector<R> phi_new((long)g.p->n_phases * cells), mu_new((long)g.p->n_solutes * cells),
      f_new((long)L.q * cells);
  Macro<R> m;
  phase_field_update(g, k, s, t, phi_new);
  macroscopic(g, L, k, s, &phi_new, t, m);
  chemical_potential_update(g, s, phi_new, m, t, mu_new);
  lattice_boltzmann_update(g, L, s, m, f_new);
  s.phi.swap(phi_new);
  s.mu.swap(mu_new);
  s.f.swap(f_new);
}

template <class R>
R objective(const Grid& g, const OracleObjective* o, const State<R>& s) {
  const OracleProblem* p = g.p;
  const int N = p->n_phases;
  const long cells = g.cells;
  R frac = 0.0;
  for (long x = 0; x < cells; ++x) {
    R ph[4];
    for (int a = 0; a < N; ++a) ph[a] = s.phi[a * cells + x];
    for (int a = 1; a < N; ++a) frac += h_fn(ph, N, a);
  }
  frac = frac / (double)cells;
  // soft-argmax of r * phi_s(r) along the +x ray from (x0, y0, z0)
  int nr = g.n[0] - o->x0;
  double mx = -1e300;
  std::vector<R> z(nr);
  for (int r = 0; r < nr; ++r) {
    z[r] = o->kappa * (double)r * s.phi[o->solid * cells + g.idx(o->x0 + r, o->y0, o->z0)];
    mx = std::max(mx, val(z[r]));
  }
  R num = 0.0, den = 0.0;
  for (int r = 0; r < nr; ++r) {
    R e = exp(z[r] - mx);
    num += (double)r * e;
    den += e;
  }
  return o->w_frac * frac + o->w_tip * (num / den) / (double)g.n[0];
}

int check(const OracleProblem* p) {
  if (!p) return -1;
  if (p->dim != 2 && p->dim != 3) return -1;
  if ((p->dim == 2 && p->q != 9) || (p->dim == 3 && p->q != 19 && p->q != 27)) return -1;
  if (p->n_phases < 2 || p->n_phases > 4 || p->n_solutes < 1 || p->n_solutes > 2) return -1;
  if (p->nx < 3 || p->ny < 3 || (p->dim == 3 && p->nz < 3)) return -1;
  for (int a = 0; a < p->n_phases; ++a)
    for (int b = 0; b < p->n_phases; ++b)
      if (p->tilt[a][b] != p->tilt[b][a]) return -1;
  return 0;
}

}  // namespace

extern "C" {

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Gradient-energy density A(q) of one pair and its derivative dA/dq, with
// the crystal axes turned by theta about z.
int oracle_gradient_energy(const double* q, int dim, double delta, double theta, double q_floor,
                           double* A, double* dA) {
  if (dim != 2 && dim != 3) return -1;
  const double c = std::cos(theta), sn = std::sin(theta);
  const double qr[3] = {c * q[0] + sn * q[1], -sn * q[0] + c * q[1], dim == 3 ? q[2] : 0.0};
  *A = A_value(theta == 0.0 ? q : qr, dim, delta, q_floor);
  double d = delta;
  dA_dq_tilted(q, dim, d, theta, q_floor, dA);
  return 0;
}

// The Gibbs-simplex projection step of the phase-field update [R11], on one
// vector of 1..4 values (in place).
int oracle_project_simplex(double* u, int m) {
  if (m < 1 || m > 4) return -1;
  project_simplex(u, m);
  return 0;
}

// Lattice weights w_k and velocities c_k (3 ints per direction) of the
// lattice with q directions; f = w_k is the fluid at rest with rho = 1.
int oracle_lattice(int q, double* w, int* c) {
  if (q != 9 && q != 19 && q != 27) return -1;
  Lattice L = make_lattice(q);
  for (int k = 0; k < q; ++k) {
    if (w) w[k] = L.w[k];
    if (c)
      for (int a = 0; a < 3; ++a) c[3 * k + a] = L.c[k][a];
  }
  return 0;
}

// Advance (phi, mu, f) in place by n_steps steps, the first at time n0.
int oracle_run(const OracleProblem* p, long n0, int n_steps, double* phi, double* mu, double* f) {
  if (check(p)) return -1;
  Grid g(p);
  Lattice L = make_lattice(p->q);
  Coeffs<double> k = plain_coeffs<double>(p);
  State<double> s;
  s.phi.assign(phi, phi + (long)p->n_phases * g.cells);
  s.mu.assign(mu, mu + (long)p->n_solutes * g.cells);
  s.f.assign(f, f + (long)L.q * g.cells);
  for (int n = 0; n < n_steps; ++n) step(g, L, k, s, n0 + n);
  std::memcpy(phi, s.phi.data(), sizeof(double) * s.phi.size());
  std::memcpy(mu, s.mu.data(), sizeof(double) * s.mu.size());
  std::memcpy(f, s.f.data(), sizeof(double) * s.f.size());
  return 0;
}

// Moving frame of the directional-solidification case (the window follows
// the growth front).  Moves the state `rows` cells down the vertical axis
// (y in 2D, z in 3D): layer v takes the values of layer v + rows and the top
// `rows` layers repeat the old top layer (a zero-gradient far field).  The
// caller lowers v0 by `rows`, so that the frozen temperature stays with the
// material.  Needs 0 <= rows < n_vertical and no obstacle rows on that axis.
int oracle_shift_frame(const OracleProblem* p, int rows, double* phi, double* mu, double* f) {
  if (check(p)) return -1;
  Grid g(p);
  const int ax = p->dim == 3 ? 2 : 1;
  const int nv = g.n[ax];
  if (rows < 0 || rows >= nv || p->wall_rows[ax] > 0) return -1;
  auto shift = [&](double* a, int planes) {
    for (int pl = 0; pl < planes; ++pl) {
      double* b = a + (long)pl * g.cells;
      const std::vector<double> old(b, b + g.cells);
      for (long i = 0; i < g.cells; ++i) {
        int c[3];
        g.coords(i, c);
        int from[3] = {c[0], c[1], c[2]};
        from[ax] = std::min(c[ax] + rows, nv - 1);
        b[i] = old[g.idx(from[0], from[1], from[2])];
      }
    }
  };
  shift(phi, p->n_phases);
  shift(mu, p->n_solutes);
  shift(f, p->q);
  return 0;
}

// Derived fields at time n: c (K-1 planes), rho, U (dim planes).
int oracle_derived(const OracleProblem* p, long n, const double* phi, const double* mu,
                   const double* f, double* c_out, double* rho_out, double* u_out) {
  if (check(p)) return -1;
  Grid g(p);
  Lattice L = make_lattice(p->q);
  Coeffs<double> k = plain_coeffs<double>(p);
  State<double> s;
  s.phi.assign(phi, phi + (long)p->n_phases * g.cells);
  s.mu.assign(mu, mu + (long)p->n_solutes * g.cells);
  s.f.assign(f, f + (long)L.q * g.cells);
  Macro<double> m;
  macroscopic(g, L, k, s, static_cast<const std::vector<double>*>(nullptr), (double)n, m);
  for (long x = 0; x < g.cells; ++x) {
    double ph[4], mm[2];
    for (int a = 0; a < p->n_phases; ++a) ph[a] = phi[a * g.cells + x];
    for (int i = 0; i < p->n_solutes; ++i) mm[i] = mu[i * g.cells + x];
    int cx[3];
    g.coords(x, cx);
    const double T = temperature(p, g.vertical(cx), (double)n);
    for (int i = 0; i < p->n_solutes; ++i) {
      double cc = 0.0;
      for (int a = 0; a < p->n_phases; ++a) cc += h_fn(ph, p->n_phases, a) * c_phase(p, a, i, mm, T);
      if (c_out) c_out[i * g.cells + x] = cc;
    }
    if (rho_out) rho_out[x] = m.rho[x];
    if (u_out)
      for (int a = 0; a < p->dim; ++a) u_out[a * g.cells + x] = m.u[a * g.cells + x];
  }
  return 0;
}

// Global totals in FP64: out[0] = sum_x sum_k f_k, out[1..K-1] = sum_x c_i,
// out[K] = mean_x sum_{a>0} h_a.  Each cell's value is formed first, then
// the cells are added sequentially in index order.
int oracle_invariants(const OracleProblem* p, long n, const double* phi, const double* mu,
                      const double* f, double* out) {
  if (check(p)) return -1;
  Grid g(p);
  const int N = p->n_phases, NC = p->n_solutes, Q = p->q;
  double mass = 0.0, sol[2] = {0.0, 0.0}, frac = 0.0;
  for (long x = 0; x < g.cells; ++x) {
    double ph[4], mm[2];
    for (int a = 0; a < N; ++a) ph[a] = phi[a * g.cells + x];
    for (int i = 0; i < NC; ++i) mm[i] = mu[i * g.cells + x];
    double rho = 0.0;
    for (int q = 0; q < Q; ++q) rho += f[q * g.cells + x];
    mass += rho;
    int cx[3];
    g.coords(x, cx);
    const double T = temperature(p, g.vertical(cx), (double)n);
    for (int i = 0; i < NC; ++i) {
      double cc = 0.0;
      for (int a = 0; a < N; ++a) cc += h_fn(ph, N, a) * c_phase(p, a, i, mm, T);
      sol[i] += cc;
    }
    double hs = 0.0;
    for (int a = 1; a < N; ++a) hs += h_fn(ph, N, a);
    frac += hs;
  }
  out[0] = mass;
  for (int i = 0; i < NC; ++i) out[1 + i] = sol[i];
  out[1 + NC] = frac / (double)g.cells;
  return 0;
}

// Objective after n_steps from the given state, and its exact directional
// derivative along (dmu0, dcoef) by forward-mode dual numbers.
//   dcoef[0]: tangent of the interface mobility 1/tau_phi
//   dcoef[1]: tangent of the anisotropy strength of every pair with delta != 0
//   dcoef[2]: tangent of g*beta_c for solute 0
int oracle_objective(const OracleProblem* p, const OracleObjective* o, long n0, int n_steps,
                     const double* phi, const double* mu, const double* f, const double* dmu0,
                     const double* dcoef, double* J, double* dJ) {
  if (check(p)) return -1;
  Grid g(p);
  Lattice L = make_lattice(p->q);
  Coeffs<Dual> k;
  k.inv_tau_phi = Dual(1.0 / p->tau_phi, dcoef ? dcoef[0] : 0.0);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      k.delta[a][b] = Dual(p->delta[a][b], (dcoef && p->delta[a][b] != 0.0) ? dcoef[1] : 0.0);
  k.gbeta_c[0] = Dual(p->gbeta_c[0], dcoef ? dcoef[2] : 0.0);
  k.gbeta_c[1] = Dual(p->gbeta_c[1], 0.0);
  State<Dual> s;
  const long cells = g.cells;
  s.phi.resize((long)p->n_phases * cells);
  s.mu.resize((long)p->n_solutes * cells);
  s.f.resize((long)L.q * cells);
  for (long i = 0; i < (long)s.phi.size(); ++i) s.phi[i] = Dual(phi[i], 0.0);
  for (long i = 0; i < (long)s.mu.size(); ++i) s.mu[i] = Dual(mu[i], dmu0 ? dmu0[i] : 0.0);
  for (long i = 0; i < (long)s.f.size(); ++i) s.f[i] = Dual(f[i], 0.0);
  for (int n = 0; n < n_steps; ++n) step(g, L, k, s, n0 + n);
  Dual j = objective(g, o, s);
  *J = j.v;
  if (dJ) *dJ = j.d;
  return 0;
}

// Jacobian-vector product of n_steps steps: the state after n_steps and
// its exact tangent along the initial-state tangent (dphi, dmu, df, each
// NULL for zero) and the parameter tangent dcoef (as in oracle_objective),
// by forward-mode dual numbers.  Outputs: t_phi, t_mu, t_f (N, K-1 and Q
// planes of the tangent of the final state; any may be NULL).
int oracle_tangent(const OracleProblem* p, long n0, int n_steps, const double* phi, const double* mu,
                   const double* f, const double* dphi, const double* dmu, const double* df,
                   const double* dcoef, double* t_phi, double* t_mu, double* t_f) {
  if (check(p)) return -1;
  Grid g(p);
  Lattice L = make_lattice(p->q);
  Coeffs<Dual> k;
  k.inv_tau_phi = Dual(1.0 / p->tau_phi, dcoef ? dcoef[0] : 0.0);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      k.delta[a][b] = Dual(p->delta[a][b], (dcoef && p->delta[a][b] != 0.0) ? dcoef[1] : 0.0);
  k.gbeta_c[0] = Dual(p->gbeta_c[0], dcoef ? dcoef[2] : 0.0);
  k.gbeta_c[1] = Dual(p->gbeta_c[1], 0.0);
  State<Dual> s;
  const long cells = g.cells;
  s.phi.resize((long)p->n_phases * cells);
  s.mu.resize((long)p->n_solutes * cells);
  s.f.resize((long)L.q * cells);
  for (long i = 0; i < (long)s.phi.size(); ++i) s.phi[i] = Dual(phi[i], dphi ? dphi[i] : 0.0);
  for (long i = 0; i < (long)s.mu.size(); ++i) s.mu[i] = Dual(mu[i], dmu ? dmu[i] : 0.0);
  for (long i = 0; i < (long)s.f.size(); ++i) s.f[i] = Dual(f[i], df ? df[i] : 0.0);
  for (int n = 0; n < n_steps; ++n) step(g, L, k, s, n0 + n);
  if (t_phi)
    for (long i = 0; i < (long)s.phi.size(); ++i) t_phi[i] = s.phi[i].d;
  if (t_mu)
    for (long i = 0; i < (long)s.mu.size(); ++i) t_mu[i] = s.mu[i].d;
  if (t_f)
    for (long i = 0; i < (long)s.f.size(); ++i) t_f[i] = s.f[i].d;
  return 0;
}

// Plain-double objective of a given state (for finite differences).
int oracle_objective_value(const OracleProblem* p, const OracleObjective* o, const double* phi,
                           double* J) {
  if (check(p)) return -1;
  Grid g(p);
  State<double> s;
  s.phi.assign(phi, phi + (long)p->n_phases * g.cells);
  *J = objective(g, o, s);
  return 0;
}

// Floating-point operations of n_steps steps from the given state, by stage
// (out[0] phase field, out[1] moments and forces, out[2] chemical potential,
// out[3] lattice Boltzmann): the same steps as oracle_run on the counting
// number type, with one thread so that the tally is exact.
int oracle_count_flops(const OracleProblem* p, long n0, int n_steps, const double* phi,
                       const double* mu, const double* f, double* out) {
  if (check(p)) return -1;
  Grid g(p);
  Lattice L = make_lattice(p->q);
  Coeffs<Cnt> k = plain_coeffs<Cnt>(p);
  State<Cnt> s;
  s.phi.assign(phi, phi + (long)p->n_phases * g.cells);
  s.mu.assign(mu, mu + (long)p->n_solutes * g.cells);
  s.f.assign(f, f + (long)L.q * g.cells);
#ifdef _OPENMP
  const int threads = omp_get_max_threads();
  omp_set_num_threads(1);
#endif
  for (int j = 0; j < 4; ++j) out[j] = 0.0;
  for (int n = 0; n < n_steps; ++n) {
    const double t = (double)(n0 + n);
    std::vector<Cnt> phi_new((long)p->n_phases * g.cells), mu_new((long)p->n_solutes * g.cells),
        f_new((long)L.q * g.cells);
    Macro<Cnt> m;
    long long c0 = g_flops;
    phase_field_update(g, k, s, t, phi_new);
    long long c1 = g_flops;
    macroscopic(g, L, k, s, &phi_new, t, m);
    long long c2 = g_flops;
    chemical_potential_update(g, s, phi_new, m, t, mu_new);
    long long c3 = g_flops;
    lattice_boltzmann_update(g, L, s, m, f_new);
    long long c4 = g_flops;
    out[0] += (double)(c1 - c0);
    out[1] += (double)(c2 - c1);
    out[2] += (double)(c3 - c2);
    out[3] += (double)(c4 - c3);
    s.phi.swap(phi_new);
    s.mu.swap(mu_new);
    s.f.swap(f_new);
  }
#ifdef _OPENMP
  omp_set_num_threads(threads);
#endif
  return 0;
}

}  // extern "C"

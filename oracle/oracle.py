"""ORACLE loader -- test infrastructure only.

ctypes front end of ``gpflbm_oracle.cpp``, the plain FP64 CPU statement of the
coupled Grand-Potential phase-field / lattice-Boltzmann time step (Sec. 2 and
Algorithm 1 of the paper).  Only the test suite, the package's smoke check
and the CPU-baseline leg of the benchmark import this module; the product
path never does.  Nothing here touches the CUDA library.

A *scenario* is the plain dict built by the seeded input generator (grid,
boundary conditions, material parameters); this module turns it into the
oracle's own problem struct.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gpflbm_oracle.cpp")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libgpflbm_oracle.so")


def build(force=False):
    """Compile the oracle with the host C++ compiler (FP64, no FMA contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


class OracleProblem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dim", ctypes.c_int), ("q", ctypes.c_int),
        ("n_phases", ctypes.c_int), ("n_solutes", ctypes.c_int),
        ("bc", ctypes.c_int * 3), ("wall_rows", ctypes.c_int * 3),
        ("tau_f", ctypes.c_double), ("tau_phi", ctypes.c_double), ("eps", ctypes.c_double),
        ("gamma", (ctypes.c_double * 4) * 4), ("delta", (ctypes.c_double * 4) * 4),
        ("A", ctypes.c_double * 4), ("ceq", (ctypes.c_double * 2) * 4), ("S", ctypes.c_double * 4),
        ("D_liq", ctypes.c_double), ("a_at", ctypes.c_double),
        ("h_drag", ctypes.c_double), ("W0", ctypes.c_double),
        ("gbeta_c", ctypes.c_double * 2), ("c_ref", ctypes.c_double * 2),
        ("gbeta_T", ctypes.c_double), ("T_ref", ctypes.c_double),
        ("T_E", ctypes.c_double), ("undercool", ctypes.c_double),
        ("G", ctypes.c_double), ("V", ctypes.c_double), ("v0", ctypes.c_double),
        ("q_floor", ctypes.c_double),
        ("eta", ctypes.c_double * 4),
        ("tilt", (ctypes.c_double * 4) * 4),
        ("dceq_dT", (ctypes.c_double * 2) * 4),
    ]


class OracleObjective(ctypes.Structure):
    _fields_ = [
        ("w_frac", ctypes.c_double), ("w_tip", ctypes.c_double), ("kappa", ctypes.c_double),
        ("x0", ctypes.c_int), ("y0", ctypes.c_int), ("z0", ctypes.c_int), ("solid", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(OracleProblem)
        O = ctypes.POINTER(OracleObjective)
        L.oracle_run.argtypes = [P, ctypes.c_long, ctypes.c_int, dp, dp, dp]
        L.oracle_shift_frame.argtypes = [P, ctypes.c_int, dp, dp, dp]
        L.oracle_count_flops.argtypes = [P, ctypes.c_long, ctypes.c_int, dp, dp, dp, dp]
        L.oracle_derived.argtypes = [P, ctypes.c_long, dp, dp, dp, dp, dp, dp]
        L.oracle_invariants.argtypes = [P, ctypes.c_long, dp, dp, dp, dp]
        L.oracle_objective.argtypes = [P, O, ctypes.c_long, ctypes.c_int, dp, dp, dp, dp, dp, dp, dp]
        L.oracle_objective_value.argtypes = [P, O, dp, dp]
        L.oracle_tangent.argtypes = [P, ctypes.c_long, ctypes.c_int, dp, dp, dp, dp, dp, dp, dp, dp,
                                     dp, dp]
        L.oracle_lattice.argtypes = [ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int)]
        L.oracle_gradient_energy.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, dp,
                                             dp]
        L.oracle_project_simplex.argtypes = [dp, ctypes.c_int]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n):
    lib().oracle_set_threads(int(n))


def max_threads():
    return int(lib().oracle_max_threads())


def problem(sc):
    """Oracle problem struct from a scenario dict (grid + parameters)."""
    g, pr = sc["grid"], sc["params"]
    p = OracleProblem()
    p.nx, p.ny, p.nz = g["nx"], g["ny"], g.get("nz", 1)
    p.dim = 3 if g.get("nz", 1) > 1 else 2
    p.q = g.get("lattice") or (19 if p.dim == 3 else 9)
    p.n_phases, p.n_solutes = sc["n_phases"], sc["n_solutes"]
    for a in range(3):
        p.bc[a] = g["bc"][a]
        p.wall_rows[a] = g["wall_rows"][a]
    for name in ("tau_f", "tau_phi", "eps", "D_liq", "a_at", "h_drag", "W0", "gbeta_T", "T_ref",
                 "T_E", "undercool", "G", "V", "v0", "q_floor"):
        setattr(p, name, float(pr[name]))
    for a in range(4):
        p.A[a] = pr["A"][a]
        p.S[a] = pr["S"][a]
        for b in range(4):
            p.gamma[a][b] = pr["gamma"][a][b]
            p.delta[a][b] = pr["delta"][a][b]
        for i in range(2):
            p.ceq[a][i] = pr["ceq"][a][i]
    for i in range(2):
        p.gbeta_c[i] = pr["gbeta_c"][i]
        p.c_ref[i] = pr["c_ref"][i]
    for a in range(4):
        p.eta[a] = pr.get("eta_rho", [0.0] * 4)[a]
        for b in range(4):
            p.tilt[a][b] = pr.get("tilt", [[0.0] * 4] * 4)[a][b]
        for i in range(2):
            p.dceq_dT[a][i] = pr.get("dceq_dT", [[0.0] * 2] * 4)[a][i]
    return p


def lattice(q):
    w = np.zeros(q)
    c = np.zeros(3 * q, dtype=np.int32)
    assert lib().oracle_lattice(q, _dp(w), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int))) == 0
    return w, c.reshape(q, 3)


def project_simplex(v):
    """The oracle's Euclidean projection of v (1..4 values) onto the simplex
    {sum = 1, u >= 0}, the last step of the phase-field update."""
    u = np.array(v, dtype=np.float64)
    assert lib().oracle_project_simplex(_dp(u), len(u)) == 0
    return u


def gradient_energy(q, delta, q_floor=1e-12, theta=0.0):
    """(A(q), dA/dq) of the pairwise gradient-energy density, crystal axes
    turned by theta about z."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    A = ctypes.c_double()
    dA = np.zeros(len(q))
    assert lib().oracle_gradient_energy(_dp(q), len(q), float(delta), float(theta), float(q_floor),
                                        ctypes.byref(A), _dp(dA)) == 0
    return A.value, dA


def rest_populations(sc):
    """f_k = w_k (fluid at rest, rho = 1) as Q planes of the grid."""
    p = problem(sc)
    w, _ = lattice(p.q)
    cells = p.nx * p.ny * (p.nz if p.dim == 3 else 1)
    return np.repeat(w[:, None], cells, axis=1).reshape(-1).copy()


def run(sc, phi, mu, f, n_steps, n0=0):
    """Advance copies of (phi, mu, f) by n_steps; returns the new arrays (FP64)."""
    p = problem(sc)
    phi = np.ascontiguousarray(phi, dtype=np.float64).copy()
    mu = np.ascontiguousarray(mu, dtype=np.float64).copy()
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    rc = lib().oracle_run(ctypes.byref(p), int(n0), int(n_steps), _dp(phi), _dp(mu), _dp(f))
    if rc != 0:
        raise ValueError("oracle_run rejected the problem")
    return phi, mu, f


def count_flops(sc, phi, mu, f, n_steps=1, n0=0):
    """Floating-point operations per cell-update of the method (the oracle's
    own steps on a counting number type), by stage: dict of phase_field,
    macroscopic, chemical_potential, lattice_boltzmann and total."""
    p = problem(sc)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(4)
    if lib().oracle_count_flops(ctypes.byref(p), int(n0), int(n_steps), _dp(phi), _dp(mu), _dp(f),
                                _dp(out)) != 0:
        raise ValueError("oracle_count_flops rejected the problem")
    cells = p.nx * p.ny * (p.nz if p.dim == 3 else 1)
    per = out / float(cells * n_steps)
    names = ("phase_field", "macroscopic", "chemical_potential", "lattice_boltzmann")
    d = dict(zip(names, per))
    d["total"] = float(per.sum())
    return d


def shift_frame(sc, phi, mu, f, rows):
    """Moving frame: the state moved `rows` cells down the vertical axis, the
    top layers repeating the old top layer (copies; the caller lowers v0 by
    `rows`)."""
    p = problem(sc)
    phi = np.array(phi, dtype=np.float64)
    mu = np.array(mu, dtype=np.float64)
    f = np.array(f, dtype=np.float64)
    if lib().oracle_shift_frame(ctypes.byref(p), int(rows), _dp(phi), _dp(mu), _dp(f)) != 0:
        raise ValueError("oracle_shift_frame rejected the problem or the shift")
    return phi, mu, f


def derived(sc, phi, mu, f, n=0):
    """(c, rho, U) at time n from the state."""
    p = problem(sc)
    cells = p.nx * p.ny * (p.nz if p.dim == 3 else 1)
    c = np.zeros(p.n_solutes * cells)
    rho = np.zeros(cells)
    u = np.zeros(p.dim * cells)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    rc = lib().oracle_derived(ctypes.byref(p), int(n), _dp(phi), _dp(mu), _dp(f), _dp(c), _dp(rho),
                              _dp(u))
    if rc != 0:
        raise ValueError("oracle_derived rejected the problem")
    return c, rho, u


def invariants(sc, phi, mu, f, n=0):
    """(mass, [solute_i], solid fraction) of the state at time n as plain
    sequential FP64 sums."""
    p = problem(sc)
    out = np.zeros(2 + p.n_solutes)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert lib().oracle_invariants(ctypes.byref(p), int(n), _dp(phi), _dp(mu), _dp(f), _dp(out)) == 0
    return out[0], out[1:1 + p.n_solutes].copy(), out[1 + p.n_solutes]


def objective_spec(obj):
    o = OracleObjective()
    o.w_frac, o.w_tip, o.kappa = obj["w_frac"], obj["w_tip"], obj["kappa"]
    o.x0, o.y0, o.z0 = obj["x0"], obj["y0"], obj.get("z0", 0)
    o.solid = obj.get("solid", 1)
    return o


def objective(sc, obj, phi, mu, f, n_steps, dmu0=None, dcoef=None, n0=0):
    """J after n_steps and its exact directional derivative (forward-mode duals)."""
    p = problem(sc)
    o = objective_spec(obj)
    J = ctypes.c_double()
    dJ = ctypes.c_double()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    dm = None if dmu0 is None else np.ascontiguousarray(dmu0, dtype=np.float64)
    dc = None if dcoef is None else np.ascontiguousarray(dcoef, dtype=np.float64)
    rc = lib().oracle_objective(ctypes.byref(p), ctypes.byref(o), int(n0), int(n_steps), _dp(phi),
                                _dp(mu), _dp(f), _dp(dm), _dp(dc), ctypes.byref(J), ctypes.byref(dJ))
    if rc != 0:
        raise ValueError("oracle_objective rejected the problem")
    return J.value, dJ.value


def objective_value(sc, obj, phi):
    """J of a given state (N phase planes, liquid first), without stepping."""
    p = problem(sc)
    o = objective_spec(obj)
    J = ctypes.c_double()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    if lib().oracle_objective_value(ctypes.byref(p), ctypes.byref(o), _dp(phi), ctypes.byref(J)) != 0:
        raise ValueError("oracle_objective_value rejected the problem")
    return J.value


def tangent(sc, phi, mu, f, n_steps, dphi=None, dmu=None, df=None, dcoef=None, n0=0):
    """Jacobian-vector product of n_steps steps (forward-mode duals): the
    tangent (phi, mu, f planes) of the state after n_steps along the initial
    tangent (dphi, dmu, df; None = 0) and the parameter tangent dcoef
    (1/tau_phi, delta, g beta_c)."""
    p = problem(sc)
    cells = p.nx * p.ny * (p.nz if p.dim == 3 else 1)
    arr = [np.ascontiguousarray(a, dtype=np.float64) for a in (phi, mu, f)]
    tan = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (dphi, dmu, df, dcoef)]
    out = (np.zeros(p.n_phases * cells), np.zeros(p.n_solutes * cells), np.zeros(p.q * cells))
    rc = lib().oracle_tangent(ctypes.byref(p), int(n0), int(n_steps), *[_dp(a) for a in arr],
                              *[_dp(a) for a in tan], *[_dp(a) for a in out])
    if rc != 0:
        raise ValueError("oracle_tangent rejected the problem")
    return out

"""Seeded synthetic scenarios: grids, material parameters and initial states.

This module builds inputs only; it holds none of the time-step arithmetic.
The CUDA library and the FP64 oracle are both fed from it, so the parity
tests compare the two on identical arrays.

Five workloads, named after what they are:

* ``dendrite2d``  -- binary alloy, single dendrite, 128 x 128, D2Q9, FP64,
  periodic in x, two obstacle rows at each end of y, seed radius 6.
* ``eutectic2d``  -- binary eutectic (liquid, alpha, beta), 1024 x 512,
  D2Q9, FP32, alpha/beta lamellae 16 cells wide in the bottom 32 rows, frozen
  temperature gradient G = 1e-4 pulled at V = 1e-3, solutal + thermal
  buoyancy.
* ``dendrite3d``  -- binary dendrite, 256^3, D3Q19, FP32 (or 16-bit
  populations), walls on every axis, sphere radius 8.
* ``eutectic3d``  -- ternary eutectic (liquid + three solids, two solutes),
  256 x 256 x 512, D3Q19, FP32, Voronoi patches of mean diameter 12 in the
  bottom 24 layers, G = 1e-4, V = 5e-4.
* ``adjoint2d``   -- the dendrite on 512 x 512 in FP32 (differentiation).

Parameter readings (lattice units, dx = dt = 1):

* interface width eps = 4 cells (the paper's eps/dx = 48/12 = 20/5 = 4);
* interface energies gamma = 1/dx of the paper's gamma = 1: 1/12 for the
  dendrites (dx = 12) and 1/5 for the eutectics (dx = 5);
* liquid diffusivity D dt/dx^2: 2.88/144 = 0.02 (dendrites), 1/25 = 0.04
  (eutectics);
* phase-field relaxation tau_phi = 4 d gamma (twice the explicit
  stability bound of the isotropic two-phase equation);
* temperature coupling S_a = 2 A_a |c_l^eq - c_a^eq|^2, so that a melt at
  mu = 0 and undercooling u is the melt at supersaturation u;
* drag: h = 2.757, W0 = eps;
* antitrapping coefficient a_at = pi^2/16: for the current
  -a_at eps phi_l [c_l - c_a] (dphi_a/dt) n_a with the mobility
  M = D phi_l / (2 A) and h_l = phi_l^2 (3 - 2 phi_l) on the obstacle
  profile, the solute balance across a slowly moving planar interface
  leaves a chemical-potential jump proportional to
  int (h_l / phi_l - Theta) dxi - a_at eps = (pi^2/16 - a_at) eps
  (thin-interface analysis of the one-sided model), so pi^2/16 removes the
  solute trapping of order V eps / D; the pi/4 of the obstacle-potential
  literature belongs to a current weighted differently;
* the eutectics' isotherm T = T_E sits theta0 / G above the top of the
  initial solid, theta0 the front undercooling at which that solid grows
  at about V under the model's capillarity (oracle runs of one lamella
  pair and of a 32 x 32 patch crop: theta0 = 0.125 for the 16-cell
  lamellae at V = 1e-3, 0.064 for the patches at V = 5e-4).  With the
  isotherm at the solid's top the solid melts back: the curvature of
  16-cell lamellae at gamma = 1/5 needs about 0.06 of undercooling to
  stand still, and G = 1e-4 gives 0.05 over the whole 512-row grid.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014) keyed on
(seed, stream, index), so any sub-range of a grid can be regenerated alone.
"""
import math

import numpy as np

PERIODIC, WALL = 0, 1
MASK64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 finaliser applied to uint64 counters (numpy, vectorised)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, stream, index):
    """U[0, 1) doubles for the given counters (53-bit mantissas)."""
    key = np.uint64(((int(seed) * 0x100000001B3) ^ (int(stream) << 40)) & MASK64)
    with np.errstate(over="ignore"):
        z = splitmix64(np.asarray(index, dtype=np.uint64) ^ key)
        z = splitmix64(z)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _blank_params():
    z4 = [[0.0] * 4 for _ in range(4)]
    return {
        "tau_f": 0.8, "tau_phi": 1.0, "eps": 4.0,
        "gamma": [row[:] for row in z4], "delta": [row[:] for row in z4],
        "A": [1.0] * 4, "ceq": [[0.0, 0.0] for _ in range(4)], "S": [0.0] * 4,
        # antitrapping: pi^2/16 cancels the chemical-potential jump of the
        # obstacle profile for this current (liquid-weighted, divided by the
        # mobility D phi_l / (2 A)), see the module docstring
        "D_liq": 0.02, "a_at": math.pi ** 2 / 16.0, "h_drag": 2.757, "W0": 4.0,
        "gbeta_c": [0.0, 0.0], "c_ref": [0.0, 0.0], "gbeta_T": 0.0, "T_ref": 1.0,
        "T_E": 1.0, "undercool": 0.0, "G": 0.0, "V": 0.0, "v0": 0.0,
        "q_floor": 1e-12,
        "eta_rho": [0.0] * 4,  # shrinkage (rho_a - rho_l) / rho_l per phase; off unless set
        "tilt": [row[:] for row in z4],  # crystal axes of a pair turned about z (radians)
        "dceq_dT": [[0.0, 0.0] for _ in range(4)],  # ceq_a(T) = ceq_a + dceq_dT_a (T - T_E)
    }


def _set_thermo(p, n_phases, n_solutes, ceq, gamma, delta_sl, dim):
    for a in range(n_phases):
        for i in range(n_solutes):
            p["ceq"][a][i] = float(ceq[a][i])
    for a in range(n_phases):
        for b in range(n_phases):
            if a != b:
                p["gamma"][a][b] = float(gamma)
                if a == 0 or b == 0:
                    p["delta"][a][b] = float(delta_sl)
    for a in range(1, n_phases):
        d2 = sum((p["ceq"][0][i] - p["ceq"][a][i]) ** 2 for i in range(n_solutes))
        p["S"][a] = 2.0 * p["A"][a] * d2
    p["tau_phi"] = 4.0 * dim * gamma
    p["W0"] = p["eps"]


WORKLOADS = ("dendrite2d", "eutectic2d", "dendrite3d", "eutectic3d", "adjoint2d")


def scenario(name, nx=None, ny=None, nz=None, precision=None, seed=None, **overrides):
    """Scenario dict for a named workload; sizes may be overridden (crops)."""
    p = _blank_params()
    if name in ("dendrite2d", "adjoint2d"):
        n = 128 if name == "dendrite2d" else 512
        grid = {"nx": nx or n, "ny": ny or n, "nz": 1, "bc": [PERIODIC, WALL, PERIODIC],
                "wall_rows": [0, 2, 0]}
        NP, NC = 2, 1
        p["tau_f"] = 0.8
        _set_thermo(p, NP, NC, [[0.45], [0.10]], 1.0 / 12.0, 0.02, 2)
        p["D_liq"] = 0.02
        p["undercool"] = 0.3
        p["gbeta_c"] = [1e-5, 0.0]
        p["c_ref"] = [0.45, 0.0]
        init = {"kind": "seed", "radius": 6.0, "noise": 1e-4}
        prec = "fp64" if name == "dendrite2d" else "fp32"
        steps = 1000 if name == "dendrite2d" else 500
    elif name == "eutectic2d":
        grid = {"nx": nx or 1024, "ny": ny or 512, "nz": 1, "bc": [PERIODIC, WALL, PERIODIC],
                "wall_rows": [0, 0, 0]}
        NP, NC = 3, 1
        p["tau_f"] = 0.7
        _set_thermo(p, NP, NC, [[0.5], [0.2], [0.8]], 1.0 / 5.0, 0.0, 2)
        p["D_liq"] = 0.04
        p["G"], p["V"] = 1e-4, 1e-3
        p["v0"] = 32.0 + 0.125 / p["G"]  # the front 0.125 below T_E
        p["gbeta_c"] = [1e-5, 0.0]
        p["c_ref"] = [0.5, 0.0]
        p["gbeta_T"], p["T_ref"] = 1e-5, 1.0
        init = {"kind": "lamellae", "width": 16, "height": 32, "c0": [0.5], "noise": 1e-3}
        prec, steps = "fp32", 20000
    elif name == "dendrite3d":
        n = 256
        grid = {"nx": nx or n, "ny": ny or n, "nz": nz or n, "bc": [WALL, WALL, WALL],
                "wall_rows": [0, 0, 0]}
        NP, NC = 2, 1
        p["tau_f"] = 0.8
        _set_thermo(p, NP, NC, [[0.45], [0.10]], 1.0 / 12.0, 0.02, 3)
        p["D_liq"] = 0.02
        p["undercool"] = 0.3
        p["gbeta_c"] = [1e-5, 0.0]
        p["c_ref"] = [0.45, 0.0]
        init = {"kind": "seed", "radius": 8.0, "noise": 1e-4}
        prec, steps = "fp32", 5000
    elif name == "eutectic3d":
        grid = {"nx": nx or 256, "ny": ny or 256, "nz": nz or 512,
                "bc": [PERIODIC, PERIODIC, WALL], "wall_rows": [0, 0, 0]}
        NP, NC = 4, 2
        p["tau_f"] = 0.7
        third = 1.0 / 3.0
        _set_thermo(p, NP, NC, [[third, third], [0.8, 0.1], [0.1, 0.8], [0.1, 0.1]], 1.0 / 5.0,
                    0.0, 3)
        p["D_liq"] = 0.04
        p["G"], p["V"] = 1e-4, 5e-4
        p["v0"] = 24.0 + 0.064 / p["G"]  # the front 0.064 below T_E
        p["gbeta_c"] = [1e-5, 1e-5]
        p["c_ref"] = [third, third]
        init = {"kind": "voronoi", "diameter": 12.0, "height": 24, "c0": [third, third],
                "noise": 0.0}
        prec, steps = "fp32", 10000
    else:
        raise ValueError("unknown workload %r" % (name,))
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(k)
        p[k] = v
    return {
        "name": name, "grid": grid, "n_phases": NP, "n_solutes": NC, "params": p,
        "precision": precision or prec, "init": init,
        "seed": 1000 + WORKLOADS.index(name) if seed is None else seed,
        "steps": steps,
    }


def dims(sc):
    g = sc["grid"]
    return g["nx"], g["ny"], g.get("nz", 1)


def cells(sc):
    nx, ny, nz = dims(sc)
    return nx * ny * nz


def _coords(sc):
    nx, ny, nz = dims(sc)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1), y.reshape(-1), z.reshape(-1)


def _seed_profile(r, radius, eps):
    """Solid fraction of a round seed: the flat-interface obstacle profile
    0.5 (1 - sin(4 (r - R) / (pi eps))) across |r - R| < pi^2 eps / 8."""
    half = math.pi ** 2 * eps / 8.0
    s = 0.5 * (1.0 - np.sin(4.0 * np.clip(r - radius, -half, half) / (math.pi * eps)))
    return s


def _voronoi_phase(sc, x, y):
    nx, ny, _ = dims(sc)
    init = sc["init"]
    n_seeds = max(3, int(round(nx * ny / (math.pi * (init["diameter"] / 2.0) ** 2))))
    sx = uniform(sc["seed"], 11, np.arange(n_seeds)) * nx
    sy = uniform(sc["seed"], 12, np.arange(n_seeds)) * ny
    ph = 1 + np.minimum((uniform(sc["seed"], 13, np.arange(n_seeds)) * 3).astype(np.int64), 2)
    best = np.full(x.shape, np.inf)
    owner = np.zeros(x.shape, dtype=np.int64)
    for s in range(n_seeds):
        dx = np.abs(x + 0.5 - sx[s])
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(y + 0.5 - sy[s])
        dy = np.minimum(dy, ny - dy)
        d2 = dx * dx + dy * dy
        closer = d2 < best
        best = np.where(closer, d2, best)
        owner = np.where(closer, s, owner)
    return ph[owner]


def initial_state(sc):
    """(phi, mu): N phase planes (liquid first) and K-1 chemical-potential
    planes, float64, SoA with x fastest."""
    nx, ny, nz = dims(sc)
    n = nx * ny * nz
    NP, NC = sc["n_phases"], sc["n_solutes"]
    p, init = sc["params"], sc["init"]
    x, y, z = _coords(sc)
    phi = np.zeros((NP, n))
    if init["kind"] == "seed":
        cx, cy, cz = nx / 2.0, ny / 2.0, nz / 2.0
        if nz > 1:
            r = np.sqrt((x + 0.5 - cx) ** 2 + (y + 0.5 - cy) ** 2 + (z + 0.5 - cz) ** 2)
        else:
            r = np.sqrt((x + 0.5 - cx) ** 2 + (y + 0.5 - cy) ** 2)
        phi[1] = _seed_profile(r, init["radius"], p["eps"])
        phi[0] = 1.0 - phi[1]
        noise = init["noise"] * (2.0 * uniform(sc["seed"], 1, np.arange(n)) - 1.0)
        mu = noise[None, :].repeat(NC, axis=0)
    elif init["kind"] == "lamellae":
        vert = y if nz == 1 else z
        solid = vert < init["height"]
        which = 1 + (x // init["width"]) % 2
        for a in (1, 2):
            phi[a] = (solid & (which == a)).astype(np.float64)
        phi[0] = 1.0 - phi[1] - phi[2]
        mu = np.zeros((NC, n))
        for i in range(NC):
            c = init["c0"][i] + init["noise"] * (2.0 * uniform(sc["seed"], 2 + i, np.arange(n)) - 1.0)
            mu[i] = 2.0 * p["A"][0] * (c - p["ceq"][0][i])
    elif init["kind"] == "voronoi":
        solid = z < init["height"]
        plane = _voronoi_phase(sc, x[: nx * ny], y[: nx * ny])
        which = np.tile(plane, nz)
        for a in range(1, NP):
            phi[a] = (solid & (which == a)).astype(np.float64)
        phi[0] = 1.0 - phi[1:].sum(axis=0)
        mu = np.zeros((NC, n))
        for i in range(NC):
            c = init["c0"][i]
            if init["noise"]:
                c = c + init["noise"] * (2.0 * uniform(sc["seed"], 2 + i, np.arange(n)) - 1.0)
            mu[i] = 2.0 * p["A"][0] * (c - p["ceq"][0][i])
    else:
        raise ValueError(init["kind"])
    return phi.reshape(-1).copy(), mu.reshape(-1).copy()

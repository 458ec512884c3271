"""Helpers of the GPU parity tests: run the CUDA library and the FP64 oracle
on the same seeded input and measure per-field relative L-infinity errors,
e(X) = max|X_gpu - X_ref| / max(max|X_ref|, 1e-30)."""
import numpy as np

from oracle import oracle
from paper_2608_26908_gb300 import gpflbm, inputs


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(float(np.abs(ref).max()), 1e-30)
    return float(np.abs(got - ref).max()) / scale


def reference(sc, steps, phi0=None, mu0=None, f0=None):
    if phi0 is None:
        phi0, mu0 = inputs.initial_state(sc)
    if f0 is None:
        f0 = oracle.rest_populations(sc)
    phi, mu, f = oracle.run(sc, phi0, mu0, f0, steps)
    c, rho, u = oracle.derived(sc, phi, mu, f, steps)
    NP, NC = sc["n_phases"], sc["n_solutes"]
    q = sc["grid"].get("lattice") or (19 if sc["grid"].get("nz", 1) > 1 else 9)
    w, _ = oracle.lattice(q)
    f = f.reshape(q, -1)
    return {"phi": phi.reshape(NP, -1), "mu": mu.reshape(NC, -1), "c": c.reshape(NC, -1),
            "rho": rho.reshape(1, -1), "u": u.reshape(len(u) // len(rho), -1),
            "f": f, "dev": f - w[:, None]}


def device_run(sc, steps, phi0=None, mu0=None, f0=None, chunks=None):
    if phi0 is None:
        phi0, mu0 = inputs.initial_state(sc)
    sim = gpflbm.Sim(sc)
    sim.set_state(phi0, mu0, f0)
    for n in (chunks or [steps]):
        sim.step(n)
    out = sim.fields(("phi", "mu", "c", "f", "rho", "u"))
    out["dev"] = sim.deviations()
    return sim, out


def errors(sc, steps, **kw):
    ref = reference(sc, steps)
    sim, got = device_run(sc, steps, **kw)
    errs = {k: rel_err(got[k], ref[k]) for k in ("phi", "mu", "c", "rho", "u", "dev")}
    return errs, sim, got, ref

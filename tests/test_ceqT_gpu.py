"""Temperature-dependent equilibrium compositions ceq_a(T) with the
temperature term of Eq. conc on the GPU against the oracle.

Every phase and solute gets its own slope dceq/dT under a fast-falling
frozen temperature (G = 4e-3, V = 2e-2); the step then runs the
extended-model kernel table.  Element-by-element parity after 100 steps
with the plain step's tolerances; the FP64 solute totals are conserved and
equal the oracle's at the same time; a uniform melt follows the closed form.
"""
import numpy as np
import pytest

from oracle import oracle
from parity import errors
from paper_2608_26908_gb300 import gpflbm, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5, "fp32_f16": 2e-3, "fp32_bf16": 5e-3}
SLOPES = [[0.4, -0.2], [0.1, 0.3], [-0.3, 0.05], [0.2, 0.2]]

CASES = [
    ("eutectic2d", dict(nx=200, ny=90), "fp64"),
    ("eutectic2d", dict(nx=200, ny=90), "fp32"),
    ("dendrite2d", dict(), "fp32"),
    ("dendrite2d", dict(nx=70, ny=50), "fp32_f16"),
    ("eutectic3d", dict(nx=36, ny=34, nz=40), "fp32"),
    ("eutectic3d", dict(nx=36, ny=34, nz=40), "fp64"),
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp32"),
    ("dendrite3d", dict(nx=40, ny=36, nz=33, lattice=27), "fp32"),
]


def _case(name, size, prec, slopes=SLOPES):
    size = dict(size)
    lattice = size.pop("lattice", None)
    sc = inputs.scenario(name, precision=prec, **size)
    if lattice:
        sc["grid"]["lattice"] = lattice
    if name == "eutectic3d":
        sc["init"]["height"] = 12
    pr = sc["params"]
    pr["G"], pr["V"] = 4e-3, 2e-2
    if name.startswith("eutectic"):  # the isotherm near the solid's top
        pr["v0"] = 32.0 if name == "eutectic2d" else 24.0
    pr["dceq_dT"] = [row[:] for row in slopes]
    return sc


def _tol(prec, field):
    return 1e-8 if prec == "fp64" and field in ("u", "dev") else TOL[prec]


@pytest.mark.parametrize("name,size,prec", CASES)
def test_ceqT_parity_100_steps(name, size, prec):
    errs, sim, got, ref = errors(_case(name, size, prec), 100)
    print("%s/%s %s" % (name, prec, " ".join("%s=%.2e" % kv for kv in sorted(errs.items()))))
    for k, e in errs.items():
        if k == "dev" and prec.startswith("fp32_"):
            continue  # stored populations are rounded to 16 bits
        assert e <= _tol(prec, k), (k, e)


def test_extended_model_all_at_once():
    """ceq(T), turned crystal axes and shrinkage together, FP64."""
    sc = _case("eutectic2d", dict(nx=120, ny=70), "fp64")
    NP = sc["n_phases"]
    sc["params"]["tilt"] = [[0.4 if a < NP and b < NP and (a == 0) != (b == 0) else 0.0
                             for b in range(4)] for a in range(4)]
    sc["params"]["eta_rho"] = [0.0, 0.2, 0.1, 0.0]
    errs, _, _, _ = errors(sc, 100)
    for k, e in errs.items():
        assert e <= _tol("fp64", k), (k, e)


@pytest.mark.parametrize("name,size", [("eutectic2d", dict(nx=120, ny=70)),
                                       ("eutectic3d", dict(nx=24, ny=22, nz=30))])
def test_ceqT_solute_is_conserved_and_matches_the_oracle(name, size):
    sc = _case(name, size, "fp64")
    sc["params"]["gbeta_c"] = [3e-3, 2e-3]  # strong flow
    phi0, mu0 = inputs.initial_state(sc)
    sim = gpflbm.Sim(sc)
    sim.set_state(phi0, mu0)
    _, s0, _, _ = sim.invariants()
    sim.step(60)
    _, s1, _, _ = sim.invariants()
    np.testing.assert_allclose(s1, s0, rtol=1e-12)
    fld = sim.fields(("phi", "mu"))
    _, s_ref, _ = oracle.invariants(sc, fld["phi"], fld["mu"], sim.fields(("f",))["f"], 60)
    np.testing.assert_allclose(s1, s_ref, rtol=1e-12)


def test_uniform_melt_follows_the_falling_temperature():
    """All liquid at rest: mu rises by 2 A k G V per step (closed form)."""
    sc = inputs.scenario("dendrite2d", nx=40, ny=30, precision="fp64")
    sc["grid"]["wall_rows"] = [0, 0, 0]
    pr = sc["params"]
    pr["gbeta_c"] = [0.0, 0.0]
    pr["G"], pr["V"] = 4e-3, 1e-2
    pr["dceq_dT"][0][0] = 0.5
    cells = 40 * 30
    phi = np.concatenate([np.ones(cells), np.zeros(cells)])
    mu = np.full(cells, 0.02)
    sim = gpflbm.Sim(sc)
    sim.set_state(phi, mu)
    sim.step(50)
    got = sim.fields(("mu",))["mu"]
    np.testing.assert_allclose(got, 0.02 + 50 * 2 * pr["A"][0] * 0.5 * 4e-3 * 1e-2, rtol=0, atol=1e-13)

"""Shrinkage force (Eq. shrinkage) on the GPU against the oracle.

Every solid phase is given the paper's density ratio eta = (1.2 - 1)/1 = 0.2;
the kernels then take the collision after the phase-field update (the force
needs phi^{n+1}).  Element-by-element parity after 100 steps with the
tolerances of the plain step (test_parity_gpu): FP64 1e-10 (U and the
population deviations 1e-8), FP32 1e-5.
"""
import numpy as np
import pytest

from parity import errors
from paper_2608_26908_gb300 import gpflbm, inputs

pytestmark = pytest.mark.gpu

ETA = 0.2
TOL = {"fp64": 1e-10, "fp32": 1e-5}

CASES = [
    ("dendrite2d", dict(), "fp64"),
    ("dendrite2d", dict(), "fp32"),
    ("eutectic2d", dict(nx=200, ny=90), "fp32"),
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp32"),
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp64"),
    ("eutectic3d", dict(nx=36, ny=34, nz=40), "fp32"),
    ("dendrite3d", dict(nx=40, ny=36, nz=33, lattice=27), "fp32"),
]


def _case(name, size, prec, eta=ETA):
    size = dict(size)
    lattice = size.pop("lattice", None)
    sc = inputs.scenario(name, precision=prec, **size)
    if lattice:
        sc["grid"]["lattice"] = lattice
    if name == "eutectic3d":
        sc["init"]["height"] = 12
    sc["params"]["eta_rho"] = [0.0] + [eta if a < sc["n_phases"] else 0.0 for a in range(1, 4)]
    return sc


def _tol(prec, field):
    return 1e-8 if prec == "fp64" and field in ("u", "dev") else TOL[prec]


@pytest.mark.parametrize("name,size,prec", CASES)
def test_shrinkage_parity_100_steps(name, size, prec):
    errs, sim, got, ref = errors(_case(name, size, prec), 100)
    print("%s/%s %s" % (name, prec, " ".join("%s=%.2e" % kv for kv in sorted(errs.items()))))
    for k, e in errs.items():
        assert e <= _tol(prec, k), (k, e)


def test_shrinkage_changes_the_flow():
    """The same run with and without the density ratio: the populations part
    ways (the shrinkage variant of the kernel is the one that ran)."""
    res = []
    for eta in (0.0, ETA):
        sc = _case("dendrite2d", {}, "fp64", eta=eta)
        sc["params"]["gbeta_c"] = [0.0, 0.0]  # shrinkage alone drives the flow
        sim = gpflbm.Sim(sc)
        sim.set_state(*inputs.initial_state(sc))
        sim.step(40)
        res.append(sim.deviations())
    assert np.abs(res[0]).max() < 1e-14  # at rest without shrinkage or buoyancy
    assert np.abs(res[1]).max() > 1e-7


def test_adjoint_rejects_shrinkage():
    sc = _case("adjoint2d", dict(nx=40, ny=36), "fp32")
    sim = gpflbm.Sim(sc)
    sim.set_state(*inputs.initial_state(sc))
    obj = {"w_frac": 1.0, "w_tip": 0.0, "kappa": 1.0, "x0": 20, "y0": 18}
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.adjoint(obj, 4, 2)
    assert e.value.status == gpflbm.ERR_UNSUPPORTED

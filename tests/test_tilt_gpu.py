"""Turned crystal axes (the seed misorientation theta of the dendrite cases)
on the GPU against the oracle.

The solid-liquid pairs of every case get the tilt; the step then runs the
turned-axes kernel table.  Element-by-element parity after 100 steps with the
tolerances of the plain step (test_parity_gpu): FP64 1e-10 (U and the
population deviations 1e-8), FP32 1e-5; with FP16 / BF16 population storage
the macroscopic fields within 2e-3 / 5e-3.
"""
import math

import numpy as np
import pytest

from parity import errors
from paper_2608_26908_gb300 import gpflbm, inputs

pytestmark = pytest.mark.gpu

THETA = 0.3
TOL = {"fp64": 1e-10, "fp32": 1e-5, "fp32_f16": 2e-3, "fp32_bf16": 5e-3}

CASES = [
    ("dendrite2d", dict(), "fp64"),
    ("dendrite2d", dict(), "fp32"),
    ("dendrite2d", dict(nx=70, ny=50), "fp32_f16"),
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp32_bf16"),
    ("eutectic2d", dict(nx=200, ny=90), "fp32"),
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp32"),
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp64"),
    ("eutectic3d", dict(nx=36, ny=34, nz=40), "fp32"),
    ("dendrite3d", dict(nx=40, ny=36, nz=33, lattice=27), "fp32"),
]


def _case(name, size, prec, theta=THETA):
    size = dict(size)
    lattice = size.pop("lattice", None)
    sc = inputs.scenario(name, precision=prec, **size)
    if lattice:
        sc["grid"]["lattice"] = lattice
    if name == "eutectic3d":
        sc["init"]["height"] = 12
    NP = sc["n_phases"]
    sc["params"]["tilt"] = [[theta if a < NP and b < NP and (a == 0) != (b == 0) else 0.0
                             for b in range(4)] for a in range(4)]
    return sc


def _tol(prec, field):
    return 1e-8 if prec == "fp64" and field in ("u", "dev") else TOL[prec]


@pytest.mark.parametrize("name,size,prec", CASES)
def test_tilt_parity_100_steps(name, size, prec):
    errs, sim, got, ref = errors(_case(name, size, prec), 100)
    print("%s/%s %s" % (name, prec, " ".join("%s=%.2e" % kv for kv in sorted(errs.items()))))
    for k, e in errs.items():
        if k == "dev" and prec.startswith("fp32_"):
            continue  # stored populations are rounded to 16 bits
        assert e <= _tol(prec, k), (k, e)


def _phi_after(sc, steps):
    sim = gpflbm.Sim(sc)
    sim.set_state(*inputs.initial_state(sc))
    sim.step(steps)
    return sim.fields(("phi",))["phi"]


def test_tilt_turns_the_growth_and_a_quarter_turn_does_not():
    """theta = 0.3 moves the front (the turned kernel ran); theta = pi/2 is
    the untilted run up to the rounding of cos(pi/2) (cubic symmetry)."""
    base = _phi_after(_case("dendrite2d", {}, "fp64", theta=0.0), 60)
    turned = _phi_after(_case("dendrite2d", {}, "fp64"), 60)
    quarter = _phi_after(_case("dendrite2d", {}, "fp64", theta=math.pi / 2), 60)
    assert np.abs(turned - base).max() > 1e-6
    assert np.abs(quarter - base).max() < 1e-12

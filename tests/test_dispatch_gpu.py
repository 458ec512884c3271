"""How a 3D step is launched, and the two extremes of the tile dispatch.

A 3D step sends every tile whose reach is pure liquid to the lean liquid
path and every other tile to the general path: in one launch with two phases
in FP32 on D3Q19, in two launches otherwise, and not at all on slabs or with
shrinkage (every tile general).  gpflbm_step_launches reports which.  The
mixed case is covered by the parity tests of every 3D configuration; here a
grid of pure liquid (no tile general) and a grid that is interface from end
to end (no tile liquid) are compared with the oracle."""
import numpy as np
import pytest

from paper_2608_26908_gb300 import gpflbm, inputs
from parity import device_run, reference, rel_err

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
SIZE = dict(nx=40, ny=36, nz=33)


def _launches(sc, **kw):
    sim = gpflbm.Sim(sc, **kw)
    try:
        return sim.step_launches()
    finally:
        sim.close()


def test_step_launches_per_configuration():
    d3 = inputs.scenario("dendrite3d", precision="fp32", **SIZE)
    assert _launches(d3) == 1  # two phases, FP32, D3Q19: one launch for both paths
    assert _launches(inputs.scenario("dendrite3d", precision="fp32_f16", **SIZE)) == 1
    assert _launches(inputs.scenario("dendrite3d", precision="fp64", **SIZE)) == 2
    assert _launches(inputs.scenario("eutectic3d", precision="fp32", nx=36, ny=34, nz=40)) == 2
    q27 = inputs.scenario("dendrite3d", precision="fp32", **SIZE)
    q27["grid"]["lattice"] = 27
    assert _launches(q27) == 2
    shrink = inputs.scenario("dendrite3d", precision="fp32", **SIZE)
    shrink["params"]["eta_rho"][1] = 0.1
    assert _launches(shrink) == 1  # every tile takes the general path
    assert _launches(d3, slab=(0, 17)) == 1  # slabs too
    assert _launches(inputs.scenario("eutectic2d", nx=64, ny=48)) == 1


def _liquid_state(sc, amp):
    """Pure liquid everywhere; the chemical potentials carry seeded noise of
    amplitude amp so that buoyancy drives a flow."""
    n = inputs.cells(sc)
    NP, NC = sc["n_phases"], sc["n_solutes"]
    phi = np.zeros((NP, n))
    phi[0] = 1.0
    rng = np.random.default_rng(11)
    mu = amp * (2.0 * rng.random((NC, n)) - 1.0)
    return phi.reshape(-1), mu.reshape(-1)


@pytest.mark.parametrize("name", ["dendrite3d", "eutectic3d"])
def test_all_liquid_grid_takes_only_the_liquid_path(name):
    size = SIZE if name == "dendrite3d" else dict(nx=36, ny=34, nz=40)
    sc = inputs.scenario(name, precision="fp32", **size)
    sc["params"]["gbeta_c"] = [2e-2, 1e-2]
    phi0, mu0 = _liquid_state(sc, 0.05)
    ref = reference(sc, 20, phi0, mu0)
    sim, got = device_run(sc, 20, phi0, mu0)
    sim.close()
    assert np.array_equal(got["phi"], ref["phi"])  # exactly the pure-liquid values
    for k in ("mu", "c", "rho", "u", "dev"):
        assert rel_err(got[k], ref[k]) <= TOL32, (k, rel_err(got[k], ref[k]))
    assert float(np.abs(ref["u"]).max()) > 1e-7  # the flow the test is about


def test_grid_with_no_liquid_tile():
    """A dendrite seed that fills a small box: every tile's reach holds the
    interface, so the liquid path takes nothing (one launch, general pass
    only)."""
    sc = inputs.scenario("dendrite3d", precision="fp32", nx=24, ny=20, nz=14)
    sc["init"]["radius"] = 7.0
    sc["params"]["gbeta_c"] = [2e-3, 0.0]
    ref = reference(sc, 20)
    sim, got = device_run(sc, 20)
    sim.close()
    for k in ("phi", "mu", "c", "rho", "u", "dev"):
        assert rel_err(got[k], ref[k]) <= TOL32, (k, rel_err(got[k], ref[k]))

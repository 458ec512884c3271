"""Slab decomposition on one GPU: a 3D grid split along its vertical axis
into slabs (gpflbm_create_slab), each stepped after the halo exchange
(gpflbm_halo_pack / gpflbm_halo_unpack, the messages copied on the device),
gives bit for bit the single-domain step's fields on every plane, and the
slabs' totals add up to the whole grid's."""
import numpy as np
import pytest

from paper_2608_26908_gb300 import gpflbm, inputs, slabs

pytestmark = pytest.mark.gpu


def _run_both(sc, parts, steps):
    phi0, mu0 = inputs.initial_state(sc)
    nx, ny, nz = inputs.dims(sc)
    layer = nx * ny
    NP, NC = sc["n_phases"], sc["n_solutes"]
    whole = gpflbm.Sim(sc)
    whole.set_state(phi0, mu0)
    whole.step(steps)
    ref = whole.fields(("phi", "mu", "f"))
    ref["dev"] = whole.deviations()
    runs = []
    for r, (v0, n) in enumerate(parts):
        sim = gpflbm.Sim(sc, slab=(v0, n))
        sl = phi0.reshape(NP, nz * layer)[:, v0 * layer:(v0 + n) * layer].reshape(-1)
        sm = mu0.reshape(NC, nz * layer)[:, v0 * layer:(v0 + n) * layer].reshape(-1)
        sim.set_state(sl, sm)
        runs.append(slabs.Slab(sim, r, len(parts)))
    for _ in range(steps):
        slabs.step_all(runs)
    return whole, ref, runs, layer


@pytest.mark.parametrize("name,size,prec,parts,steps,extra", [
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp32", [(0, 17), (17, 16)], 40, {}),
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp64", [(0, 10), (10, 11), (21, 12)], 30, {}),
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp32_f16", [(0, 2), (2, 29), (31, 2)], 25, {}),
    ("eutectic3d", dict(nx=36, ny=34, nz=40), "fp32", [(0, 21), (21, 19)], 30, {}),
    ("eutectic3d", dict(nx=36, ny=34, nz=40), "fp32", [(0, 13), (13, 14), (27, 13)], 20, {"lattice": 27}),
    ("dendrite3d", dict(nx=40, ny=36, nz=33), "fp32", [(0, 16), (16, 17)], 20, {"tilt": 0.3}),
])
def test_slabs_match_the_whole_grid_bit_for_bit(name, size, prec, parts, steps, extra):
    sc = inputs.scenario(name, precision=prec, **size)
    if name == "eutectic3d":
        sc["init"]["height"] = 12
    sc["params"]["gbeta_c"] = [2e-3, 1e-3]  # a flow across the slab boundaries
    if "lattice" in extra:
        sc["grid"]["lattice"] = extra["lattice"]
    if "tilt" in extra:
        sc["params"]["tilt"][0][1] = sc["params"]["tilt"][1][0] = extra["tilt"]
    whole, ref, runs, layer = _run_both(sc, parts, steps)
    tot = [0.0, np.zeros(sc["n_solutes"]), 0.0]
    for (v0, n), run in zip(parts, runs):
        got = run.sim.fields(("phi", "mu", "f"))
        got["dev"] = run.sim.deviations()
        for k in ("phi", "mu", "f", "dev"):
            want = ref[k][:, v0 * layer:(v0 + n) * layer]
            assert np.array_equal(got[k], want), (k, v0, n, float(np.abs(got[k] - want).max()))
        assert run.sim.time() == whole.time() == steps
        m, s, fr, _ = run.sim.invariants()
        tot[0] += m
        tot[1] += s
        tot[2] += fr * n * layer
    m, s, fr, _ = whole.invariants()
    cells = inputs.cells(sc)
    assert tot[0] == pytest.approx(m, rel=1e-13)
    np.testing.assert_allclose(tot[1], s, rtol=1e-12)
    assert tot[2] / cells == pytest.approx(fr, rel=1e-12, abs=1e-15)


def test_slab_needs_the_exchange_and_refuses_what_it_cannot_do():
    sc = inputs.scenario("dendrite3d", nx=24, ny=20, nz=16)
    phi0, mu0 = inputs.initial_state(sc)
    layer = 24 * 20
    sim = gpflbm.Sim(sc, slab=(0, 8))
    sim.set_state(phi0.reshape(2, -1)[:, :8 * layer].reshape(-1), mu0[:8 * layer])
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.step(1)  # no halo from the slab above yet
    assert e.value.status == gpflbm.ERR_STATE
    import torch
    msg = torch.empty(sim.halo_bytes(), dtype=torch.uint8, device="cuda")
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.halo_pack(0, msg)  # a wall below
    assert e.value.status == gpflbm.ERR_ARG
    sim.halo_pack(1, msg)
    sim.halo_unpack(1, msg)
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.step(2)  # one step per exchange
    assert e.value.status == gpflbm.ERR_ARG
    sim.step(1)
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.step(1)  # the halo was used up
    assert e.value.status == gpflbm.ERR_STATE
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.shift_frame(1)
    assert e.value.status == gpflbm.ERR_UNSUPPORTED
    for bad, status in (((0, 1), gpflbm.ERR_ARG), ((10, 7), gpflbm.ERR_ARG)):
        with pytest.raises(gpflbm.GpflbmError) as e:
            gpflbm.Sim(sc, slab=bad)
        assert e.value.status == status
    sc2 = inputs.scenario("dendrite2d", nx=24, ny=20)
    with pytest.raises(gpflbm.GpflbmError) as e:
        gpflbm.Sim(sc2, slab=(0, 8))
    assert e.value.status == gpflbm.ERR_UNSUPPORTED
    sc3 = inputs.scenario("eutectic3d", nx=24, ny=20, nz=16)
    sc3["grid"]["bc"][2] = gpflbm.PERIODIC
    with pytest.raises(gpflbm.GpflbmError) as e:
        gpflbm.Sim(sc3, slab=(0, 8))
    assert e.value.status == gpflbm.ERR_UNSUPPORTED

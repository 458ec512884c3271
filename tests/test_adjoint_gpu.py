"""Adjoint of the coupled step (gpflbm_adjoint) on the GPU.

Pins, from independent sides:
  * the oracle's forward-mode dual numbers: exact directional derivatives of
    the same discrete map in FP64 (the oracle shares no code with the GPU);
  * FP64 central finite differences of the GPU forward, step 1e-6, on a
    64 x 64 crop: the gradient within 1e-4 relative;
  * properties at the full 512 x 512, 500-step, K = 50 workload: the final
    state equals plain stepping bit for bit, J equals the oracle's J of that
    final state, dJ/dmu0 vanishes in the frozen wall rows.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_2608_26908_gb300 import gpflbm, inputs

pytestmark = pytest.mark.gpu


def _case(nx, ny, prec, ext="plain"):
    sc = inputs.scenario("adjoint2d", nx=nx, ny=ny, precision=prec)
    sc["init"]["radius"] = 6.0
    pr = sc["params"]
    pr["gbeta_c"] = [2e-3, 0.0]  # a flow strong enough to matter
    if ext == "tilt":
        pr["tilt"][0][1] = pr["tilt"][1][0] = 0.35
    elif ext == "ceqT":  # ceq(T) under a falling temperature
        pr["G"], pr["V"], pr["v0"] = 4e-3, 2e-2, 10.0
        pr["dceq_dT"][0][0], pr["dceq_dT"][1][0] = 0.4, 0.1
    return sc


def _obj(sc):
    g = sc["grid"]
    return {"w_frac": 1.0, "w_tip": 1.0, "kappa": 2.0, "x0": g["nx"] // 2, "y0": g["ny"] // 2,
            "solid": 1}


def _gpu_adjoint(sc, horizon, K):
    phi0, mu0 = inputs.initial_state(sc)
    sim = gpflbm.Sim(sc)
    sim.set_state(phi0, mu0)
    J, dpar, dmu = sim.adjoint(_obj(sc), horizon, K)
    return sim, J, dpar, dmu.astype(np.float64)


def _oracle_directional(sc, horizon, dmu0=None, dcoef=None):
    phi0, mu0 = inputs.initial_state(sc)
    f0 = oracle.rest_populations(sc)
    return oracle.objective(sc, _obj(sc), phi0, mu0, f0, horizon, dmu0=dmu0, dcoef=dcoef)


def _close(a, b, rtol, scale):
    return abs(a - b) <= rtol * max(abs(b), scale)


@pytest.mark.parametrize("ext", ["plain", "tilt", "ceqT"])
@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-8), ("fp32", 2e-4)])
def test_adjoint_matches_oracle_dual_derivatives(prec, rtol, ext):
    """40 x 36 (ragged against 256-thread blocks), 23 steps, K = 5: four
    full segments and a ragged one; the plain model, tilted crystal axes
    (0.35 rad), and temperature-dependent ceq under a falling temperature."""
    sc = _case(40, 36, prec, ext)
    H, K = 23, 5
    _, J, dpar, dmu = _gpu_adjoint(sc, H, K)
    rng = np.random.default_rng(11)
    v = rng.normal(size=dmu.shape)
    Jo, dJo = _oracle_directional(sc, H, dmu0=v)
    assert _close(J, Jo, rtol, 0.0)
    g = float(np.dot(v, dmu))
    assert _close(g, dJo, rtol, 1e-3 * float(np.abs(v * dmu).sum())), (g, dJo)
    # single cells at the interface and in the bulk liquid
    for cell in (18 * 40 + 26, 18 * 40 + 14, 3 * 40 + 5):
        e = np.zeros_like(v)
        e[cell] = 1.0
        _, dJc = _oracle_directional(sc, H, dmu0=e)
        assert _close(dmu[cell], dJc, rtol, 1e-3 * float(np.abs(dmu).max())), (cell, dmu[cell], dJc)
    for j in range(3):
        dc = np.zeros(3)
        dc[j] = 1.0
        _, dJp = _oracle_directional(sc, H, dcoef=dc)
        assert _close(dpar[j], dJp, rtol, 0.0), (j, dpar[j], dJp)


def test_adjoint_matches_central_differences_fp64():
    """64 x 64 crop, 40 steps, K = 8; FP64 central differences of the GPU
    forward with step 1e-6 (direction of unit RMS for mu0)."""
    sc = _case(64, 64, "fp64")
    H, K, h = 40, 8, 1e-6
    phi0, mu0 = inputs.initial_state(sc)
    sim, J, dpar, dmu = _gpu_adjoint(sc, H, K)
    obj = _obj(sc)

    def J_of(sc2, mu):
        s = gpflbm.Sim(sc2)
        s.set_state(phi0, mu)
        return s.adjoint(obj, H, K)[0]

    v = np.random.default_rng(3).normal(size=mu0.shape)
    fd = (J_of(sc, mu0 + h * v) - J_of(sc, mu0 - h * v)) / (2 * h)
    assert float(np.dot(v, dmu)) == pytest.approx(fd, rel=1e-4)
    base = (1.0 / sc["params"]["tau_phi"], sc["params"]["delta"][0][1], sc["params"]["gbeta_c"][0])
    for j in range(3):
        vals = []
        for sgn in (+1, -1):
            p = list(base)
            p[j] += sgn * h
            vals.append(J_of(gpflbm.with_parameters(sc, *p), mu0))
        fdp = (vals[0] - vals[1]) / (2 * h)
        assert dpar[j] == pytest.approx(fdp, rel=1e-4), (j, dpar[j], fdp)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpoint_spacing_and_reruns_give_identical_gradients(prec):
    """Every contribution is gathered in a fixed order and the recomputed
    states equal the stored ones bit for bit, so neither the checkpoint
    spacing (K = 1, K not dividing H, K = H, K > H) nor a rerun changes a
    bit of J or of the gradients."""
    sc = _case(40, 36, prec)
    H = 17
    ref = None
    for K in (1, 4, 17, 40, 4):
        _, J, dpar, dmu = _gpu_adjoint(sc, H, K)
        if ref is None:
            ref = (J, dpar, dmu)
            continue
        assert J == ref[0]
        assert np.array_equal(dpar, ref[1])
        assert np.array_equal(dmu, ref[2])


def test_adjoint_leaves_the_state_of_plain_stepping():
    sc = _case(48, 40, "fp32")
    phi0, mu0 = inputs.initial_state(sc)
    a = gpflbm.Sim(sc)
    a.set_state(phi0, mu0)
    a.adjoint(_obj(sc), 21, 6)
    b = gpflbm.Sim(sc)
    b.set_state(phi0, mu0)
    b.step(21)
    fa, fb = a.fields(("phi", "mu", "f")), b.fields(("phi", "mu", "f"))
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert a.time() == b.time() == 21


def test_adjoint_rejects_unsupported_and_invalid():
    sc = inputs.scenario("eutectic2d", nx=40, ny=30)
    sim = gpflbm.Sim(sc)
    sim.set_state(*inputs.initial_state(sc))
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.adjoint(_obj(sc), 4, 2)
    assert e.value.status == gpflbm.ERR_UNSUPPORTED
    sc = _case(40, 36, "fp32")
    sim = gpflbm.Sim(sc)
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.adjoint(_obj(sc), 4, 2)  # no state yet
    assert e.value.status == gpflbm.ERR_STATE
    sim.set_state(*inputs.initial_state(sc))
    bad = dict(_obj(sc), x0=40)
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.adjoint(bad, 4, 2)
    assert e.value.status == gpflbm.ERR_ARG
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.adjoint(_obj(sc), 0, 2)
    assert e.value.status == gpflbm.ERR_ARG


def test_autograd_function_returns_the_adjoint_gradients():
    import torch
    sc = _case(40, 36, "fp64")
    phi0, mu0 = inputs.initial_state(sc)
    sim = gpflbm.Sim(sc)
    mu = torch.tensor(mu0, dtype=torch.float64, device="cuda", requires_grad=True)
    pr = sc["params"]
    mob = torch.tensor(1.0 / pr["tau_phi"], dtype=torch.float64, requires_grad=True)
    dl = torch.tensor(pr["delta"][0][1], dtype=torch.float64, requires_grad=True)
    gb = torch.tensor(pr["gbeta_c"][0], dtype=torch.float64, requires_grad=True)
    F = gpflbm.GPFLBMFunction()
    J = F.apply(mu, mob, dl, gb, sim, phi0, _obj(sc), 11, 4)
    (2.0 * J).backward()
    _, J2, dpar, dmu = _gpu_adjoint(sc, 11, 4)
    assert float(J.detach()) == J2
    np.testing.assert_allclose(mu.grad.cpu().numpy(), 2.0 * dmu, rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose([mob.grad.item(), dl.grad.item(), gb.grad.item()], 2.0 * dpar,
                               rtol=1e-10)


def test_full_workload_properties():
    """512 x 512 FP32, 500 steps, checkpoints every 50 (the differentiation
    workload): final state as plain stepping, J from the oracle's objective
    of that final state, finite gradients, none in the frozen wall rows."""
    sc = inputs.scenario("adjoint2d")
    H, K = 500, 50
    phi0, mu0 = inputs.initial_state(sc)
    sim = gpflbm.Sim(sc)
    sim.set_state(phi0, mu0)
    J, dpar, dmu = sim.adjoint(_obj(sc), H, K)
    ref = gpflbm.Sim(sc)
    ref.set_state(phi0, mu0)
    ref.step(H)
    fa, fb = sim.fields(("phi", "mu")), ref.fields(("phi", "mu"))
    assert np.array_equal(fa["phi"], fb["phi"]) and np.array_equal(fa["mu"], fb["mu"])
    Jo = oracle.objective_value(sc, _obj(sc), fa["phi"].astype(np.float64))
    assert J == pytest.approx(Jo, rel=1e-12)
    assert np.all(np.isfinite(dmu)) and np.all(np.isfinite(dpar))
    assert np.abs(dmu).max() > 0.0 and np.all(dpar != 0.0)
    nx, ny = 512, 512
    rows = dmu.reshape(ny, nx)
    w = sc["grid"]["wall_rows"][1]
    assert np.all(rows[:w] == 0.0) and np.all(rows[ny - w:] == 0.0)


def test_full_workload_fp32_gradients_match_fp64():
    """At the full differentiation workload the FP32 gradients agree with the
    FP64 ones (themselves equal to the oracle's on crops) to the 1e-4 the
    gradients are held to against finite differences."""
    res = {}
    for prec in ("fp32", "fp64"):
        sc = inputs.scenario("adjoint2d", precision=prec)
        phi0, mu0 = inputs.initial_state(sc)
        sim = gpflbm.Sim(sc)
        sim.set_state(phi0, mu0)
        J, dpar, dmu = sim.adjoint(_obj(sc), 500, 50)
        res[prec] = (J, dpar, dmu.astype(np.float64))
    (J32, p32, m32), (J64, p64, m64) = res["fp32"], res["fp64"]
    assert J32 == pytest.approx(J64, rel=1e-6)
    np.testing.assert_allclose(p32, p64, rtol=1e-4)
    assert np.abs(m32 - m64).max() <= 1e-4 * np.abs(m64).max()


# ------------------------------------------------------------------ dot-product tests
def _dot_case():
    """40 x 36 FP64 dendrite with a perturbed flow field (f = w + noise), so
    that every block of the step's Jacobian is exercised."""
    sc = _case(40, 36, "fp64")
    phi0, mu0 = inputs.initial_state(sc)
    w, _ = oracle.lattice(9)
    cells = inputs.cells(sc)
    rng = np.random.default_rng(5)
    f0 = (w[:, None] * (1.0 + 1e-3 * rng.normal(size=(9, cells)))).reshape(-1)
    return sc, phi0, mu0, f0


@pytest.mark.parametrize("block,H,K", [("phase_field", 1, 1), ("chemical_potential", 1, 1),
                                       ("lattice_boltzmann", 1, 1), ("all", 3, 2)])
def test_vjp_dot_product_per_stencil(block, H, K):
    """<J v, w> = <v, J^T w> for each transposed stencil on its own: v and w
    on the phase field only, on mu only, on the populations only, and on
    everything over three steps (checkpointed).  J v comes from the oracle's
    forward-mode dual numbers (an independent code), J^T w from the GPU's
    gpflbm_vjp.  v is zero on phi where a cell is pure (0 or 1): there the
    oracle's projection and the GPU's untouched cell are two subgradients of
    the same kink.  FP64 on both sides."""
    sc, phi0, mu0, f0 = _dot_case()
    cells = inputs.cells(sc)
    rng = np.random.default_rng({"phase_field": 1, "chemical_potential": 2,
                                 "lattice_boltzmann": 3, "all": 4}[block])
    v = rng.normal(size=(11, cells))
    wt = rng.normal(size=(11, cells))
    s0 = phi0.reshape(2, cells)[1]
    v[0][(s0 <= 0.0) | (s0 >= 1.0)] = 0.0
    keep = {"phase_field": [0], "chemical_potential": [1], "lattice_boltzmann": list(range(2, 11)),
            "all": list(range(11))}[block]
    for arr in (v, wt):
        for k in range(11):
            if k not in keep:
                arr[k] = 0.0
    t_phi, t_mu, t_f = oracle.tangent(sc, phi0, mu0, f0, H, dphi=np.concatenate([-v[0], v[0]]),
                                      dmu=v[1], df=v[2:].reshape(-1))
    jv_w = (float(np.dot(wt[0], t_phi.reshape(2, cells)[1])) + float(np.dot(wt[1], t_mu)) +
            float(np.dot(wt[2:].reshape(-1), t_f)))
    sim = gpflbm.Sim(sc)
    sim.set_state(phi0, mu0, f0)
    grad, dpar = sim.vjp(wt, H, K)
    v_jtw = float(np.sum(v * grad))
    scale = float(np.abs(v * grad).sum())
    assert scale > 0.0
    assert abs(jv_w - v_jtw) <= 1e-10 * scale, (block, jv_w, v_jtw, scale)
    if block == "all":
        for j in range(3):
            dc = np.zeros(3)
            dc[j] = 1.0
            tp, tm, tf = oracle.tangent(sc, phi0, mu0, f0, H, dcoef=dc)
            want = (float(np.dot(wt[0], tp.reshape(2, cells)[1])) + float(np.dot(wt[1], tm)) +
                    float(np.dot(wt[2:].reshape(-1), tf)))
            assert dpar[j] == pytest.approx(want, rel=1e-9, abs=1e-12), (j, dpar[j], want)


def test_vjp_rejects_unsupported_and_invalid():
    sc = inputs.scenario("eutectic2d", nx=40, ny=30)
    sim = gpflbm.Sim(sc)
    sim.set_state(*inputs.initial_state(sc))
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.vjp(np.zeros((11, inputs.cells(sc))), 2, 1)
    assert e.value.status == gpflbm.ERR_UNSUPPORTED
    sc = _case(40, 36, "fp32")
    sim = gpflbm.Sim(sc)
    with pytest.raises(gpflbm.GpflbmError) as e:
        sim.vjp(np.zeros((11, inputs.cells(sc))), 2, 1)  # no state yet
    assert e.value.status == gpflbm.ERR_STATE


# ------------------------------------------------------------------ stated FD check
@pytest.mark.parametrize("prec,flow,rtol", [("fp32", "workload", 1e-4), ("fp64", "strong", 1e-6)])
def test_gradients_match_fp64_central_differences_at_the_stated_horizon(prec, flow, rtol):
    """The differentiation workload's check on its 64 x 64 crop over the
    500-step horizon with checkpoints every 50: dJ/d(1/tau_phi), dJ/d delta,
    dJ/d g beta_c and dJ/dmu0 along 8 random directions, against the oracle's
    exact directional derivatives (dual numbers through the same piecewise
    map, 500 steps) and against FP64 central differences of the GPU forward
    with step 1e-6.  A difference whose +h and -h runs differ in which cells
    are clamped or present at some step (a kink of the map inside +-h) is
    not a derivative of the branch the adjoint follows: such pairs are
    counted and reported, and every other pair must agree.  FP32 gradients
    (the configuration's arithmetic) with the workload's parameters at the
    stated 1e-4; FP64 gradients under a 200 times stronger flow at 1e-6."""
    H, K, h = 500, 50, 1e-6

    def crop(p):
        sc = inputs.scenario("adjoint2d", nx=64, ny=64, precision=p)
        if flow == "strong":
            sc["params"]["gbeta_c"] = [2e-3, 0.0]
        return sc

    sc_g, sc64 = crop(prec), crop("fp64")
    phi0, mu0 = inputs.initial_state(sc64)
    f0 = oracle.rest_populations(sc64)
    _, J, dpar, dmu = _gpu_adjoint(sc_g, H, K)
    obj = _obj(sc64)

    def J_and_masks(sc, mu):
        s = gpflbm.Sim(sc)
        s.set_state(phi0, mu)
        masks = []
        for _ in range(H):
            s.step(1)
            ph = s.fields(("phi",))["phi"][1]
            masks.append((ph == 0.0) | (ph == 1.0))
        s.set_state(phi0, mu)
        return s.adjoint(obj, H, K)[0], masks

    def fd_pair(sc_p, sc_m, mu_p, mu_m):
        (jp, mp), (jm, mm) = J_and_masks(sc_p, mu_p), J_and_masks(sc_m, mu_m)
        kinks = np.zeros(inputs.cells(sc64), dtype=bool)
        for a, b in zip(mp, mm):
            kinks |= a != b
        return (jp - jm) / (2 * h), int(kinks.sum())

    rng = np.random.default_rng(7)
    rows, cs = [], []
    for i in range(8):
        v = rng.normal(size=mu0.shape)
        fd, nk = fd_pair(sc64, sc64, mu0 + h * v, mu0 - h * v)
        exact = oracle.objective(sc64, obj, phi0, mu0, f0, H, dmu0=v)[1]
        rows.append(("mu0 dir %d" % i, float(np.dot(v, dmu)), exact, fd, nk))
        cs.append(float(np.linalg.norm(v) * np.linalg.norm(dmu)))
    base = (1.0 / sc64["params"]["tau_phi"], sc64["params"]["delta"][0][1], sc64["params"]["gbeta_c"][0])
    for j, name in enumerate(("1/tau_phi", "delta", "gbeta_c")):
        pp, pm = list(base), list(base)
        pp[j] += h
        pm[j] -= h
        fd, nk = fd_pair(gpflbm.with_parameters(sc64, *pp), gpflbm.with_parameters(sc64, *pm), mu0, mu0)
        dc = np.zeros(3)
        dc[j] = 1.0
        exact = oracle.objective(sc64, obj, phi0, mu0, f0, H, dcoef=dc)[1]
        rows.append((name, float(dpar[j]), exact, fd, nk))
    for name, adj, exact, fd, nk in rows:
        print("%s %s flow %-10s adjoint % .10e exact % .10e FD % .10e  |adj-exact| %.1e  |adj-FD| %.1e  "
              "kink cells %d" % (prec, flow, name, adj, exact, fd, abs(adj - exact) / abs(exact),
                                 abs(adj - fd) / abs(fd), nk))
    # the gradient in mu0 is held to rtol relative to its own size: a
    # direction's derivative v.g to rtol |v| |g| (Cauchy-Schwarz), which keeps
    # directions whose terms nearly cancel from asking for more than that
    for i, (name, adj, exact, fd, nk) in enumerate(rows):
        floor = cs[i] if i < 8 else 0.0
        assert abs(adj - exact) <= rtol * max(abs(exact), floor), (name, adj, exact)
        if nk == 0:
            assert abs(adj - fd) <= rtol * max(abs(fd), floor), (name, adj, fd)
    assert sum(r[4] == 0 for r in rows) >= 3, rows  # the FD check is not vacuous

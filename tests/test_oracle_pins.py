"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: a value the paper
prints (tests/golden), a closed form, an invariant, or a special case that
reduces to a textbook scheme.  A dropped term, a wrong sign or index, or a
transposed operand anywhere in the oracle fails at least one of them.
"""
import copy
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle
from paper_2608_26908_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _liquid_box(nx, ny, nz=1, bc=(0, 0, 0), n_phases=2, n_solutes=1, **params):
    """All-liquid scenario on a small box with no buoyancy unless asked."""
    sc = inputs.scenario("dendrite3d" if nz > 1 else "dendrite2d", nx=nx, ny=ny,
                         nz=nz if nz > 1 else None)
    sc["grid"]["bc"] = list(bc)
    sc["grid"]["wall_rows"] = [0, 0, 0]
    sc["n_phases"], sc["n_solutes"] = n_phases, n_solutes
    p = sc["params"]
    p["gbeta_c"] = [0.0, 0.0]
    p["gbeta_T"] = 0.0
    p["undercool"] = 0.0
    for k, v in params.items():
        p[k] = v
    cells = nx * ny * nz
    phi = np.zeros((n_phases, cells))
    phi[0] = 1.0
    mu = np.zeros((n_solutes, cells))
    return sc, phi.reshape(-1), mu.reshape(-1)


def _feq(w, c, rho, u):
    """Second-order equilibrium used only to build initial populations."""
    cu = np.einsum("ka,ax->kx", c[:, : u.shape[0]].astype(float), u)
    uu = (u * u).sum(axis=0)
    return w[:, None] * rho[None, :] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu[None, :])


# ----------------------------------------------------------------- lattices
def test_d2q9_weights_and_numbering_match_paper_table():
    w, c = oracle.lattice(9)
    for row in _golden("lattice_weights.txt"):
        if row[0] != "D2Q9":
            continue
        c2, count, num, den = int(row[1]), int(row[2]), int(row[3]), int(row[4])
        sel = [k for k in range(9) if (c[k] ** 2).sum() == c2]
        assert len(sel) == count
        for k in sel:
            assert w[k] == pytest.approx(num / den, abs=0, rel=1e-15)
    for k, cx, cy in (map(int, r) for r in _golden("d2q9_numbering.txt")):
        assert (c[k, 0], c[k, 1], c[k, 2]) == (cx, cy, 0)


def test_d3q27_weights_match_paper_table():
    """Classes of the paper's lattice table: k = 0 rest, 1-6 faces, 7-18
    edges, 19-26 corners, weights 8/27, 2/27, 1/54, 1/216."""
    w, c = oracle.lattice(27)
    ranges = {0: range(0, 1), 1: range(1, 7), 2: range(7, 19), 3: range(19, 27)}
    for row in _golden("lattice_weights.txt"):
        if row[0] != "D3Q27":
            continue
        c2, count, num, den = int(row[1]), int(row[2]), int(row[3]), int(row[4])
        sel = [k for k in range(27) if (c[k] ** 2).sum() == c2]
        assert sel == list(ranges[c2]) and len(sel) == count
        for k in sel:
            assert w[k] == pytest.approx(num / den, abs=0, rel=1e-15)
    assert len({tuple(v) for v in c}) == 27


@pytest.mark.parametrize("q", [9, 19, 27])
def test_lattice_moments_are_isotropic(q):
    w, c = oracle.lattice(q)
    D = 2 if q == 9 else 3
    wf = [Fraction(x).limit_denominator(1000) for x in w]
    assert sum(wf) == 1
    for a in range(D):
        assert sum(wf[k] * c[k, a] for k in range(q)) == 0
        for b in range(D):
            m2 = sum(wf[k] * c[k, a] * c[k, b] for k in range(q))
            assert m2 == (Fraction(1, 3) if a == b else 0)
    # fourth moment: (1/9)(d_ab d_cd + d_ac d_bd + d_ad d_bc)
    d = np.eye(D, dtype=int)
    for a in range(D):
        for b in range(D):
            for e in range(D):
                for g in range(D):
                    m4 = sum(wf[k] * c[k, a] * c[k, b] * c[k, e] * c[k, g] for k in range(q))
                    iso = Fraction(d[a, b] * d[e, g] + d[a, e] * d[b, g] + d[a, g] * d[b, e], 9)
                    assert m4 == iso
    # each direction has its opposite
    for k in range(q):
        assert any((c[j] == -c[k]).all() for j in range(q))


def test_presets_follow_appendix_b():
    tab = {(r[0], r[1]): float(r[2]) for r in _golden("appendix_b_parameters.txt")}
    den = inputs.scenario("dendrite2d")["params"]
    eut = inputs.scenario("eutectic2d")["params"]
    assert den["eps"] == pytest.approx(tab["binary", "eps"] / tab["binary", "dx"])
    assert eut["eps"] == pytest.approx(tab["eutectic", "eps"] / tab["eutectic", "dx"])
    assert den["D_liq"] == pytest.approx(
        tab["common", "D_liquid"] * tab["binary", "dt"] / tab["binary", "dx"] ** 2)
    assert eut["D_liq"] == pytest.approx(
        tab["common", "D_liquid"] * tab["eutectic", "dt"] / tab["eutectic", "dx"] ** 2)
    assert den["gamma"][0][1] == pytest.approx(tab["common", "gamma"] / tab["binary", "dx"])
    assert eut["gamma"][1][2] == pytest.approx(tab["common", "gamma"] / tab["eutectic", "dx"])
    assert den["delta"][0][1] == pytest.approx(tab["binary", "anisotropy_strength"])
    assert eut["delta"][1][2] == 0.0 and eut["delta"][0][1] == 0.0


# ----------------------------------------------------------------- interpolation
def _h_of(n_phases, phis, which):
    """h_which(phi) read back through the composition c = sum_a h_a c_a(mu)
    with mu = 0, c_which^eq = 1 and every other c^eq = 0."""
    m = phis.shape[1]
    sc, _, _ = _liquid_box(m, 3, n_phases=n_phases)
    for a in range(4):
        sc["params"]["ceq"][a] = [1.0 if a == which else 0.0, 0.0]
    phi = np.repeat(phis[:, :, None], 3, axis=2).transpose(0, 2, 1).reshape(n_phases, -1)
    mu = np.zeros(3 * m)
    f = oracle.rest_populations(sc)
    c, _, _ = oracle.derived(sc, phi.reshape(-1), mu, f)
    return c.reshape(3, m)[1]


def test_h_two_phase_is_smoothstep():
    s = np.linspace(0.0, 1.0, 41)
    hs = _h_of(2, np.stack([1 - s, s]), 1)
    np.testing.assert_allclose(hs, s * s * (3 - 2 * s), rtol=0, atol=1e-15)


@pytest.mark.parametrize("n_phases", [3, 4])
def test_h_sum_rule_vertices_and_edges(n_phases):
    rng = np.random.default_rng(7)
    pts = rng.dirichlet(np.ones(n_phases), size=64).T
    total = sum(_h_of(n_phases, pts, a) for a in range(n_phases))
    np.testing.assert_allclose(total, 1.0, rtol=0, atol=1e-14)
    eye = np.eye(n_phases)
    for a in range(n_phases):
        np.testing.assert_allclose(_h_of(n_phases, eye, a), eye[a], atol=1e-15)
    # on the a-b edge the multi-phase h reduces to the two-phase smoothstep
    s = np.linspace(0, 1, 17)
    edge = np.zeros((n_phases, 17))
    edge[0], edge[n_phases - 1] = 1 - s, s
    np.testing.assert_allclose(_h_of(n_phases, edge, n_phases - 1), s * s * (3 - 2 * s), atol=1e-15)


# ----------------------------------------------------------------- anisotropy
def test_anisotropy_is_one_plus_delta_cos4theta_in_2d():
    for delta in (0.0, 0.02, 0.05):
        for th in np.linspace(0, 2 * math.pi, 37):
            r = 0.37
            q = [r * math.cos(th), r * math.sin(th)]
            A, _ = oracle.gradient_energy(q, delta)
            assert A == pytest.approx((1 + delta * math.cos(4 * th)) ** 2 * r * r, rel=1e-13)


def test_cubic_anisotropy_special_directions_in_3d():
    d = 0.03
    for q, ac in (([1, 0, 0], 1 + d), ([1, 1, 0], 1 - d), ([1, 1, 1], 1 - 5 * d / 3)):
        q = np.array(q, float) * 0.5
        A, _ = oracle.gradient_energy(q, d)
        assert A == pytest.approx(ac * ac * (q @ q), rel=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_energy_derivative_matches_finite_difference(dim):
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.normal(size=dim)
        _, dA = oracle.gradient_energy(q, 0.04)
        h = 1e-6
        fd = np.zeros(dim)
        for j in range(dim):
            e = np.zeros(dim)
            e[j] = h
            fd[j] = (oracle.gradient_energy(q + e, 0.04)[0] - oracle.gradient_energy(q - e, 0.04)[0]) / (2 * h)
        np.testing.assert_allclose(dA, fd, rtol=1e-7, atol=1e-9)
    q = rng.normal(size=dim)
    _, dA = oracle.gradient_energy(q, 0.0)
    np.testing.assert_array_equal(dA, 2 * q)


# ------------------------------------------------------------ tilted crystal axes
def test_tilted_anisotropy_is_one_plus_delta_cos4_of_the_angle_to_the_axis():
    """Crystal axes turned by theta about z: the 2D density is
    (1 + delta cos 4(vartheta - theta))^2 |q|^2, vartheta the polar angle of q
    (a wrong sense of rotation gives cos 4(vartheta + theta) and fails)."""
    for theta in (0.3, -0.55, 1.0):
        for th in np.linspace(0, 2 * math.pi, 29):
            r = 0.41
            q = [r * math.cos(th), r * math.sin(th)]
            A, _ = oracle.gradient_energy(q, 0.05, theta=theta)
            assert A == pytest.approx((1 + 0.05 * math.cos(4 * (th - theta))) ** 2 * r * r, rel=1e-13)
    # in 3D the <100> axis in the x-y plane lies at angle theta
    d, theta = 0.03, 0.4
    q = 0.5 * np.array([math.cos(theta), math.sin(theta), 0.0])
    assert oracle.gradient_energy(q, d, theta=theta)[0] == pytest.approx((1 + d) ** 2 * 0.25, rel=1e-13)
    q = 0.5 * np.array([math.cos(theta + math.pi / 4), math.sin(theta + math.pi / 4), 0.0])
    assert oracle.gradient_energy(q, d, theta=theta)[0] == pytest.approx((1 - d) ** 2 * 0.25, rel=1e-13)
    # the z axis is untouched by a turn about z
    q = np.array([0.0, 0.0, 0.7])
    assert oracle.gradient_energy(q, d, theta=theta)[0] == pytest.approx((1 + d) ** 2 * 0.49, rel=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_tilted_gradient_energy_derivative_matches_finite_difference(dim):
    rng = np.random.default_rng(11)
    for _ in range(20):
        q = rng.normal(size=dim)
        theta = rng.uniform(-math.pi, math.pi)
        _, dA = oracle.gradient_energy(q, 0.04, theta=theta)
        h = 1e-6
        fd = np.zeros(dim)
        for j in range(dim):
            e = np.zeros(dim)
            e[j] = h
            fd[j] = (oracle.gradient_energy(q + e, 0.04, theta=theta)[0]
                     - oracle.gradient_energy(q - e, 0.04, theta=theta)[0]) / (2 * h)
        np.testing.assert_allclose(dA, fd, rtol=1e-7, atol=1e-9)


def _tilted_seed(dim, theta, delta_sign=1.0, steps=30):
    if dim == 2:
        sc = inputs.scenario("dendrite2d", nx=36, ny=36)
    else:
        sc = inputs.scenario("dendrite3d", nx=20, ny=20, nz=12)
    sc["init"]["noise"] = 0.0
    pr = sc["params"]
    pr["delta"] = [[delta_sign * v for v in row] for row in pr["delta"]]
    pr["tilt"] = [[theta if (a == 0) != (b == 0) else 0.0 for b in range(4)] for a in range(4)]
    phi, mu = inputs.initial_state(sc)
    nx, ny, nz = inputs.dims(sc)
    phi1, mu1, f1 = oracle.run(sc, phi, mu, oracle.rest_populations(sc), steps)
    shape = (nz, ny, nx)
    return (phi1.reshape((-1,) + shape), mu1.reshape((-1,) + shape),
            oracle.derived(sc, phi1, mu1, f1)[2].reshape((-1,) + shape))


@pytest.mark.parametrize("dim", [2, 3])
def test_quarter_turn_of_cubic_axes_changes_nothing(dim):
    """Cubic symmetry: axes turned by pi/2 give the untilted step."""
    a = _tilted_seed(dim, 0.0)
    b = _tilted_seed(dim, math.pi / 2)
    for x, y in zip(a, b):
        np.testing.assert_allclose(y, x, rtol=0, atol=1e-12 * max(1.0, np.abs(x).max()))


def test_eighth_turn_in_2d_flips_the_sign_of_delta():
    """cos 4(vartheta - pi/4) = -cos 4 vartheta: tilt pi/4 with delta is the
    untilted step with -delta."""
    a = _tilted_seed(2, 0.0, delta_sign=-1.0)
    b = _tilted_seed(2, math.pi / 4)
    for x, y in zip(a, b):
        np.testing.assert_allclose(y, x, rtol=0, atol=1e-12 * max(1.0, np.abs(x).max()))
    c = _tilted_seed(2, 0.0)
    assert np.abs(c[0] - b[0]).max() > 1e-6  # the anisotropy does act


@pytest.mark.parametrize("dim", [2, 3])
def test_mirror_in_x_turns_theta_into_minus_theta(dim):
    """A seed centred in a box symmetric under x -> -x: the run with tilt
    -theta is the mirror image of the run with +theta (u_x changes sign)."""
    phi_p, mu_p, u_p = _tilted_seed(dim, 0.35)
    phi_m, mu_m, u_m = _tilted_seed(dim, -0.35)
    flip = lambda a: a[..., ::-1]
    np.testing.assert_allclose(flip(phi_m), phi_p, rtol=0, atol=1e-12)
    np.testing.assert_allclose(flip(mu_m), mu_p, rtol=0, atol=1e-12)
    np.testing.assert_allclose(-flip(u_m[0]), u_p[0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(flip(u_m[1:]), u_p[1:], rtol=0, atol=1e-14)
    assert np.abs(phi_p - flip(phi_p)).max() > 1e-6  # the tilted seed is not symmetric itself


# ----------------------------------------------------------------- phase field
def _lap(a, dim):
    out = -2 * dim * a
    for ax in range(dim):
        out = out + np.roll(a, 1, axis=ax) + np.roll(a, -1, axis=ax)
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_isotropic_two_phase_step_is_textbook_allen_cahn(dim):
    """N = 2, no anisotropy, both phases present everywhere: one step of the
    multi-phase scheme is the scalar obstacle Allen-Cahn update with the
    standard 5-point (7-point) Laplacian."""
    n = 12
    sc, _, _ = _liquid_box(n, n, n if dim == 3 else 1, delta=[[0.0] * 4 for _ in range(4)],
                           undercool=0.15)
    p = sc["params"]
    grids = np.meshgrid(*[np.arange(n)] * dim, indexing="ij")
    phase = sum(np.sin(2 * math.pi * (k + 1) * g / n + 0.3 * k) for k, g in enumerate(grids))
    s = 0.5 + 0.25 * phase / dim  # in (0.25, 0.75); memory order (z,) y, x
    mu = 0.02 * np.cos(2 * math.pi * grids[0] / n)
    phi = np.stack([1 - s.reshape(-1), s.reshape(-1)])
    f = oracle.rest_populations(sc)
    phi1, _, _ = oracle.run(sc, phi.reshape(-1), mu.reshape(-1), f, 1)
    # closed-form scalar update
    g, eps, tau = p["gamma"][0][1], p["eps"], p["tau_phi"]
    A, cl, cs, S = p["A"][1], p["ceq"][0][0], p["ceq"][1][0], p["S"][1]
    dpsi = -mu * (cl - cs) + S * p["undercool"]  # psi_l - psi_s at T = T_E - u
    sm = s
    lap = _lap(sm, dim)
    expect = sm + (g * eps * lap - 8 * g / (math.pi ** 2 * eps) * (1 - 2 * sm)
                   + 3 * sm * (1 - sm) * dpsi) / (tau * eps)
    np.testing.assert_allclose(phi1.reshape(2, -1)[1], expect.reshape(-1), rtol=0, atol=1e-14)
    assert A == 1.0


def _flat_interface(eps, mu_shift=0.0, steps=2000, delta=0.0, dceq=None):
    n = int(16 * eps)
    sc, _, _ = _liquid_box(n, 3, bc=(1, 0, 0), eps=eps, W0=eps)
    p = sc["params"]
    if dceq is not None:  # (liquid, solid) slopes of ceq(T)
        p["dceq_dT"][0][0], p["dceq_dT"][1][0] = dceq
    for a in range(4):
        for b in range(4):
            p["delta"][a][b] = delta if (a != b and (a == 0 or b == 0)) else 0.0
    p["undercool"] = 0.3
    x = np.arange(n) + 0.5
    xc = n / 2
    half = math.pi ** 2 * eps / 8
    prof = 0.5 * (1 - np.sin(4 * np.clip(x - xc, -half, half) / (math.pi * eps)))  # solid left
    s = np.tile(prof, 3)
    phi = np.stack([1 - s, s]).reshape(-1)
    dc = p["ceq"][0][0] - p["ceq"][1][0]
    mu_star = 2 * p["A"][0] * dc * p["undercool"]
    if dceq is not None and mu_shift is not None:
        # psi_l = psi_s with ceq(T): mu* = (S_l - S_s) theta / (ceq_l(T) - ceq_s(T))
        theta = -p["undercool"]
        dcT = dc + (dceq[0] - dceq[1]) * theta
        mu_star = (p["S"][0] - p["S"][1]) * theta / dcT
    mu = np.full(3 * n, mu_star + (mu_shift or 0.0))
    f = oracle.rest_populations(sc)
    phi1, mu1, f1 = oracle.run(sc, phi, mu, f, steps)
    return sc, x, prof, phi1.reshape(2, 3, n)[1, 1], mu1.reshape(3, n)[1], mu_star, f1


def _crossing(x, s):
    j = np.where((s[:-1] >= 0.5) & (s[1:] < 0.5))[0][0]
    return x[j] + (s[j] - 0.5) / (s[j] - s[j + 1])


def test_flat_interface_keeps_obstacle_profile_and_converges():
    """At mu = mu* the grand potentials of solid and liquid are equal: the
    interface stays put (up to the shift from the solute released while the
    continuous profile relaxes to the discrete one) and keeps the obstacle
    profile 0.5 (1 - sin(4 x / (pi eps))) up to a second-order error."""
    errs, shifts = [], []
    for eps in (4.0, 8.0):
        sc, x, prof, s, mu, mu_star, f = _flat_interface(eps)
        shifts.append(abs(_crossing(x, s) - _crossing(x, prof)))
        errs.append(np.abs(s - prof).max())
    assert shifts[0] < 0.03 and shifts[1] < 0.01
    assert errs[0] < 2e-2
    assert errs[0] / errs[1] > 3.0  # second order in 1/eps


def test_flat_interface_equilibrium_compositions():
    sc, x, prof, s, mu, mu_star, f = _flat_interface(4.0, steps=400)
    p = sc["params"]
    c, _, _ = oracle.derived(sc, np.stack([1 - np.tile(s, 3), np.tile(s, 3)]).reshape(-1),
                             np.tile(mu, 3), f)
    c = c.reshape(3, -1)[1]
    u = p["undercool"]
    dc = p["ceq"][0][0] - p["ceq"][1][0]
    assert c[-1] == pytest.approx(p["ceq"][0][0] + dc * u, abs=1e-6)  # 0.555
    assert c[0] == pytest.approx(p["ceq"][1][0] + dc * u, abs=1e-6)   # 0.205


def test_flat_interface_with_temperature_dependent_ceq():
    """ceq_a(T) = ceq_a + k_a (T - T_E), k = (0.5, 0.1), T - T_E = -0.3: the
    interface is at rest at mu* = (S_l - S_s) theta / (ceq_l(T) - ceq_s(T))
    (0.320, not the 0.210 of k = 0), with c_l = ceq_l(T) + mu*/(2A) and
    c_s = ceq_s(T) + mu*/(2A) on either side; started at the k = 0 value of
    mu* the solid grows."""
    k = (0.5, 0.1)
    sc, x, prof, s, mu, mu_star, f = _flat_interface(4.0, steps=400, dceq=k)
    assert mu_star == pytest.approx(2 * 0.35 ** 2 * 0.3 / 0.23, rel=1e-12)
    assert abs(_crossing(x, s) - _crossing(x, prof)) < 0.03
    p = sc["params"]
    c, _, _ = oracle.derived(sc, np.stack([1 - np.tile(s, 3), np.tile(s, 3)]).reshape(-1),
                             np.tile(mu, 3), f)
    c = c.reshape(3, -1)[1]
    theta = -p["undercool"]
    assert c[-1] == pytest.approx(0.45 + k[0] * theta + mu_star / 2, abs=1e-6)  # 0.4598
    assert c[0] == pytest.approx(0.10 + k[1] * theta + mu_star / 2, abs=1e-6)   # 0.2298
    _, x, prof, s0, _, _, _ = _flat_interface(4.0, mu_shift=None, steps=200, dceq=k)
    assert _crossing(x, s0) > _crossing(x, prof) + 0.05


def test_uniform_melt_keeps_its_composition_as_the_temperature_falls():
    """The temperature term of Eq. conc: a uniform melt at rest under
    T = T_E + G (v - v0 - V t) with dceq_l/dT = k keeps c = ceq_l(T) + mu/(2A)
    fixed in every cell, so mu rises by 2 A k G V per step (exactly linear);
    the fields at time 0 and at time 50 give the same c."""
    for dim in (2, 3):
        sc, phi, mu = _liquid_box(5, 7, 4 if dim == 3 else 1, bc=(0, 1, 1), G=4e-3, V=1e-2, v0=3.0)
        p = sc["params"]
        p["dceq_dT"][0][0] = 0.5
        mu = mu + 0.02
        f = oracle.rest_populations(sc)
        phi1, mu1, f1 = oracle.run(sc, phi, mu, f, 50)
        rate = 2 * p["A"][0] * 0.5 * 4e-3 * 1e-2
        np.testing.assert_allclose(mu1, 0.02 + 50 * rate, rtol=0, atol=1e-13)
        c0, _, _ = oracle.derived(sc, phi, mu, f, 0)
        c1, _, _ = oracle.derived(sc, phi1, mu1, f1, 50)
        np.testing.assert_allclose(c1, c0, rtol=0, atol=1e-13)
        assert np.ptp(c0) > 0.005  # c varies with height, mu does not


def test_interface_moves_with_the_sign_of_the_driving_force():
    _, x, prof, s_lo, _, _, _ = _flat_interface(4.0, mu_shift=-0.05, steps=200)
    _, _, _, s_hi, _, _, _ = _flat_interface(4.0, mu_shift=+0.05, steps=200)
    x0 = _crossing(x, prof)
    assert _crossing(x, s_lo) > x0 + 0.05  # mu below mu*: the solid grows
    assert _crossing(x, s_hi) < x0 - 0.05  # mu above mu*: the solid melts


def test_no_ghost_phase_three_phase_equals_two_phase():
    sc2, _, _ = _liquid_box(40, 6, bc=(1, 0, 0), n_phases=2, undercool=0.3)
    sc3, _, _ = _liquid_box(40, 6, bc=(1, 0, 0), n_phases=3, undercool=0.3)
    for sc in (sc2, sc3):
        p = sc["params"]
        for a in range(3):
            for b in range(3):
                p["gamma"][a][b] = 0.2 if a != b else 0.0
                p["delta"][a][b] = 0.0
        p["ceq"][2] = [0.8, 0.0]
        p["S"][2] = 2 * (0.45 - 0.8) ** 2
        p["tau_phi"] = 4 * 2 * 0.2
    x = np.arange(40) + 0.5
    s = np.tile(np.clip(0.5 - (x - 20) / 10, 0, 1), 6)
    mu = np.full(240, 0.1)
    phi2 = np.stack([1 - s, s]).reshape(-1)
    phi3 = np.stack([1 - s, s, np.zeros_like(s)]).reshape(-1)
    a2, m2, _ = oracle.run(sc2, phi2, mu, oracle.rest_populations(sc2), 50)
    a3, m3, _ = oracle.run(sc3, phi3, mu, oracle.rest_populations(sc3), 50)
    a3 = a3.reshape(3, -1)
    assert (a3[2] == 0.0).all()
    np.testing.assert_allclose(a3[1], a2.reshape(2, -1)[1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(m3, m2, rtol=0, atol=1e-14)


def test_simplex_invariant_four_phases():
    sc = inputs.scenario("eutectic3d", nx=16, ny=16, nz=24)
    sc["init"]["height"] = 10
    phi, mu = inputs.initial_state(sc)
    f = oracle.rest_populations(sc)
    phi1, _, _ = oracle.run(sc, phi, mu, f, 15)
    phi1 = phi1.reshape(4, -1)
    assert phi1.min() >= 0.0
    np.testing.assert_allclose(phi1.sum(axis=0), 1.0, rtol=0, atol=1e-14)
    assert (phi1 != phi.reshape(4, -1)).any()


# ----------------------------------------------------------------- chemical potential
@pytest.mark.parametrize("dim", [2, 3])
def test_frozen_liquid_mu_is_ftcs_heat_equation(dim):
    """phi = liquid everywhere and U = 0: Eq. conc reduces to the explicit
    heat equation with diffusivity D; on a periodic box its exact solution is
    the Fourier multiplier (1 - 2 D sum_d (1 - cos k_d))^n."""
    n = 16
    steps = 25
    sc, phi, _ = _liquid_box(n, n, n if dim == 3 else 1)
    D = sc["params"]["D_liq"]
    shape = (n,) * dim
    mu0 = np.zeros(shape)
    mu0[(n // 2,) * dim] = 1e-3
    mu0 = mu0 + 1e-4 * np.cos(2 * math.pi * np.arange(n) / n)  # along x
    f = oracle.rest_populations(sc)
    _, mu1, f1 = oracle.run(sc, phi, mu0.reshape(-1), f, steps)
    ks = np.meshgrid(*[2 * math.pi * np.fft.fftfreq(n)] * dim, indexing="ij")
    mult = 1 - 2 * D * sum(1 - np.cos(k) for k in ks)
    expect = np.real(np.fft.ifftn(np.fft.fftn(mu0) * mult ** steps))
    np.testing.assert_allclose(mu1.reshape(shape), expect, rtol=0, atol=1e-17)
    np.testing.assert_allclose(f1, f, rtol=0, atol=1e-15)


# ----------------------------------------------------------------- lattice Boltzmann
def _taylor_green_rate(L, tau):
    sc, phi, mu = _liquid_box(L, L, tau_f=tau)
    w, c = oracle.lattice(9)
    x, y = np.meshgrid(np.arange(L), np.arange(L), indexing="xy")
    k = 2 * math.pi / L
    U0 = 1e-4
    u = np.stack([U0 * np.cos(k * x) * np.sin(k * y), -U0 * np.sin(k * x) * np.cos(k * y)])
    f = _feq(w, c, np.ones(L * L), u.reshape(2, -1)).reshape(-1)
    t0, t1 = 100, 300
    _, _, f = oracle.run(sc, phi, mu, f, t0)
    _, _, ua = oracle.derived(sc, phi, mu, f, t0)
    _, _, f = oracle.run(sc, phi, mu, f, t1 - t0, n0=t0)
    _, _, ub = oracle.derived(sc, phi, mu, f, t1)
    ref = u.reshape(-1)
    amps = [(ua * ref).sum() / (ref * ref).sum(), (ub * ref).sum() / (ref * ref).sum()]
    rate = -math.log(amps[1] / amps[0]) / (t1 - t0)
    nu = (tau - 0.5) / 3
    return rate / (2 * nu * k * k)


def test_taylor_green_decays_at_the_bgk_viscosity():
    r32 = _taylor_green_rate(32, 0.8)
    r64 = _taylor_green_rate(64, 0.8)
    assert abs(r32 - 1) < 1e-2
    assert abs(r64 - 1) < 3e-3
    assert abs(r32 - 1) / abs(r64 - 1) > 3.0  # second order in k


def _poiseuille(tau, H=16, steps=6000):
    F0 = 1e-6
    sc, phi, mu = _liquid_box(H, 4, bc=(1, 0, 0), tau_f=tau, gbeta_T=F0, T_ref=0.0, T_E=1.0)
    f = oracle.rest_populations(sc)
    _, _, f = oracle.run(sc, phi, mu, f, steps)
    _, rho, u = oracle.derived(sc, phi, mu, f, steps)
    uy = u.reshape(2, 4, H)[1, 2]
    return F0, (tau - 0.5) / 3, uy, rho


def test_poiseuille_between_bounce_back_walls():
    # bulk: discrete second difference is exactly -F/nu at any tau
    F0, nu, uy, rho = _poiseuille(0.8)
    d2 = uy[:-2] - 2 * uy[1:-1] + uy[2:]
    np.testing.assert_allclose(d2, -F0 / nu, rtol=1e-8)
    np.testing.assert_allclose(rho, 1.0, atol=1e-12)
    # halfway bounce-back puts the wall exactly half a cell out when
    # (tau - 1/2)^2 = 3/16, so the profile is the analytic parabola
    tau = 0.5 + math.sqrt(3.0) / 4.0
    F0, nu, uy, _ = _poiseuille(tau)
    H = len(uy)
    xs = np.arange(H) + 0.5
    exact = F0 / (2 * nu) * xs * (H - xs)
    np.testing.assert_allclose(uy, exact, rtol=1e-8)


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_body_force_accelerates_exactly(dim):
    F0 = 1e-5
    sc, phi, mu = _liquid_box(6, 6, 6 if dim == 3 else 1, gbeta_T=F0, T_ref=0.0, T_E=1.0)
    f = oracle.rest_populations(sc)
    steps = 37
    _, _, f1 = oracle.run(sc, phi, mu, f, steps)
    _, rho, u = oracle.derived(sc, phi, mu, f1, steps)
    u = u.reshape(dim, -1)
    np.testing.assert_allclose(rho, 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[dim - 1], F0 * (steps + 0.5), rtol=1e-12)
    np.testing.assert_allclose(u[: dim - 1], 0.0, atol=1e-20)


def test_drag_stops_flow_in_solid():
    """Uniform force through a box whose right half is solid: the implicit
    drag makes the velocity in the solid the terminal value F/kappa-scaled
    value far below the liquid one."""
    F0 = 1e-6
    sc, _, mu = _liquid_box(32, 4, bc=(1, 0, 0), gbeta_T=F0, T_ref=0.0, T_E=1.0)
    sc["params"]["h_drag"] = 50.0
    s = np.tile((np.arange(32) >= 16).astype(float), 4)
    phi = np.stack([1 - s, s]).reshape(-1)
    mu = np.full(128, 2 * 0.3 * 0.35)  # hold the interface near rest
    sc["params"]["undercool"] = 0.3
    f = oracle.rest_populations(sc)
    _, _, f1 = oracle.run(sc, phi, mu, f, 400)
    _, _, u = oracle.derived(sc, phi, mu, f1, 400)
    uy = u.reshape(2, 4, 32)[1, 1]
    assert uy[:12].max() > 50 * np.abs(uy[22:]).max()


def test_quiescent_isothermal_melt_stays_exactly_at_rest():
    sc, phi, _ = _liquid_box(20, 14, bc=(0, 1, 0), gbeta_c=[1e-3, 0.0], c_ref=[0.45, 0.0],
                             gbeta_T=1e-3, T_ref=1.0, T_E=1.0)
    mu = np.full(20 * 14, 2 * 1.0 * (0.45 - 0.45))
    f = oracle.rest_populations(sc)
    _, mu1, f1 = oracle.run(sc, phi, mu, f, 50)
    np.testing.assert_allclose(f1, f, rtol=0, atol=1e-15)
    _, _, u = oracle.derived(sc, phi, mu1, f1, 50)
    assert np.abs(u).max() == 0.0


# ----------------------------------------------------------------- conservation
@pytest.mark.parametrize("case", ["dendrite2d", "eutectic2d", "dendrite3d", "eutectic3d",
                                  "dendrite3d/D3Q27", "eutectic3d/D3Q27"])
def test_mass_and_solute_are_conserved(case):
    case, _, lat = case.partition("/")
    sizes = {"dendrite2d": dict(nx=40, ny=36), "eutectic2d": dict(nx=48, ny=40),
             "dendrite3d": dict(nx=14, ny=16, nz=18), "eutectic3d": dict(nx=16, ny=14, nz=20)}
    sc = inputs.scenario(case, **sizes[case])
    if lat:
        sc["grid"]["lattice"] = 27
    if case == "eutectic3d":
        sc["init"]["height"] = 8
    if case == "eutectic2d":
        sc["init"]["height"] = 12
    sc["params"]["gbeta_c"] = [3e-3, 2e-3]  # strong flow
    phi, mu = inputs.initial_state(sc)
    f = oracle.rest_populations(sc)
    m0, s0, _ = oracle.invariants(sc, phi, mu, f)
    phi1, mu1, f1 = oracle.run(sc, phi, mu, f, 40)
    m1, s1, _ = oracle.invariants(sc, phi1, mu1, f1, 40)
    _, _, u = oracle.derived(sc, phi1, mu1, f1, 40)
    assert np.abs(u).max() > 1e-6  # there is flow
    assert abs(m1 - m0) / m0 < 1e-12
    np.testing.assert_allclose(s1, s0, rtol=1e-12)


@pytest.mark.parametrize("case", ["eutectic2d", "eutectic3d"])
def test_solute_is_conserved_with_temperature_dependent_ceq(case):
    """Different slopes dceq_a/dT per phase and solute under a fast-falling
    temperature: the solute sum_a h_a c_a(mu, T) at T^n is conserved by the
    flux form with the temperature term at h^{n+1}."""
    sizes = {"eutectic2d": dict(nx=48, ny=40), "eutectic3d": dict(nx=16, ny=14, nz=20)}
    sc = inputs.scenario(case, **sizes[case])
    sc["init"]["height"] = 12 if case == "eutectic2d" else 8
    pr = sc["params"]
    pr["gbeta_c"] = [3e-3, 2e-3]
    pr["G"], pr["V"] = 4e-3, 2e-2
    pr["v0"] = 32.0 if case == "eutectic2d" else 24.0  # isotherm near the solid's top
    pr["dceq_dT"] = [[0.4, -0.2], [0.1, 0.3], [-0.3, 0.05], [0.2, 0.2]]
    phi, mu = inputs.initial_state(sc)
    f = oracle.rest_populations(sc)
    _, s0, _ = oracle.invariants(sc, phi, mu, f, 0)
    phi1, mu1, f1 = oracle.run(sc, phi, mu, f, 40)
    _, s1, _ = oracle.invariants(sc, phi1, mu1, f1, 40)
    np.testing.assert_allclose(s1, s0, rtol=1e-12)
    # the solute at time 40 counted with the temperature of time 0 is not
    # the same number: the temperature term did work
    _, s1_stale, _ = oracle.invariants(sc, phi1, mu1, f1, 0)
    assert np.abs(s1_stale - s0).max() > 1e-6 * np.abs(s0).max()


# ----------------------------------------------------------------- derivatives
def test_dual_number_derivatives_match_central_differences():
    sc = inputs.scenario("adjoint2d", nx=24, ny=24)
    sc["init"]["radius"] = 5.0
    sc["params"]["gbeta_c"] = [2e-3, 0.0]
    phi, mu = inputs.initial_state(sc)
    f = oracle.rest_populations(sc)
    obj = {"w_frac": 1.0, "w_tip": 1.0, "kappa": 2.0, "x0": 12, "y0": 12, "solid": 1}
    steps = 12
    rng = np.random.default_rng(5)
    dmu = rng.normal(size=mu.shape) * 1e-2
    J0, dJ = oracle.objective(sc, obj, phi, mu, f, steps, dmu0=dmu)
    h = 1e-6
    Jp, _ = oracle.objective(sc, obj, phi, mu + h * dmu, f, steps)
    Jm, _ = oracle.objective(sc, obj, phi, mu - h * dmu, f, steps)
    assert dJ == pytest.approx((Jp - Jm) / (2 * h), rel=1e-5)
    base = copy.deepcopy(sc)
    for j, key in enumerate(["tau_phi", "delta", "gbeta_c"]):
        dc = np.zeros(3)
        dc[j] = 1.0
        _, dJ = oracle.objective(sc, obj, phi, mu, f, steps, dcoef=dc)
        vals = []
        for sgn in (+1, -1):
            s2 = copy.deepcopy(base)
            pp = s2["params"]
            if key == "tau_phi":
                pp["tau_phi"] = 1.0 / (1.0 / pp["tau_phi"] + sgn * h)
            elif key == "delta":
                for a in range(4):
                    for b in range(4):
                        if pp["delta"][a][b] != 0.0:
                            pp["delta"][a][b] += sgn * h
            else:
                pp["gbeta_c"][0] += sgn * h
            vals.append(oracle.objective(s2, obj, phi, mu, f, steps)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert dJ == pytest.approx(fd, rel=1e-4, abs=1e-9), key


# ----------------------------------------------------------------- extra pins
@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_flow_advects_mu_by_central_differences(dim):
    """All liquid, uniform velocity U (f = f^eq(1, U), no force keeps U
    uniform): Eq. conc becomes the FTCS advection-diffusion scheme whose
    exact periodic solution is the multiplier
    1 - 2 D sum_d (1 - cos k_d) - i sum_d U_d sin k_d per step."""
    n, steps = 12, 15
    sc, phi, _ = _liquid_box(n, n, n if dim == 3 else 1)
    D = sc["params"]["D_liq"]
    q = 9 if dim == 2 else 19
    w, c = oracle.lattice(q)
    U = np.array([0.011, -0.007, 0.005][:dim])
    cells = n ** dim
    u = np.repeat(U[:, None], cells, axis=1)
    f = _feq(w, c, np.ones(cells), u).reshape(-1)
    _, _, u0 = oracle.derived(sc, phi, np.zeros(cells), f)
    Uc = u0.reshape(dim, -1)[:, 0]  # velocity on the grid (x, y[, z])
    rng = np.random.default_rng(11)
    mu0 = 1e-3 * rng.normal(size=(n,) * dim)
    _, mu1, _ = oracle.run(sc, phi, mu0.reshape(-1), f, steps)
    ks = np.meshgrid(*[2 * math.pi * np.fft.fftfreq(n)] * dim, indexing="ij")  # axes (z,) y, x
    mult = 1 - 2 * D * sum(1 - np.cos(k) for k in ks)
    for d in range(dim):
        mult = mult - 1j * Uc[d] * np.sin(ks[dim - 1 - d])
    expect = np.real(np.fft.ifftn(np.fft.fftn(mu0) * mult ** steps))
    np.testing.assert_allclose(mu1.reshape((n,) * dim), expect, rtol=0, atol=1e-15)


def test_solutal_buoyancy_sign_and_size():
    """Uniform liquid richer than c_ref: the force g beta (c_l - c_ref) acts
    upward along the vertical axis and U grows as F (n + 1/2)."""
    gb, dc = 2e-4, 0.05
    sc, phi, _ = _liquid_box(5, 6, gbeta_c=[gb, 0.0], c_ref=[0.45, 0.0])
    mu = np.full(30, 2 * 1.0 * dc)  # c_l = 0.45 + dc
    f = oracle.rest_populations(sc)
    steps = 9
    _, _, f1 = oracle.run(sc, phi, mu, f, steps)
    _, _, u = oracle.derived(sc, phi, mu, f1, steps)
    np.testing.assert_allclose(u.reshape(2, -1)[1], gb * dc * (steps + 0.5), rtol=1e-11)


def test_implicit_drag_decay_factor():
    """Uniform mushy cells (phi_l = 1/2 held by mu = mu*) with an initial
    uniform flow: F = -rho kappa U with the implicit U gives the exact decay
    factor (1 - kappa/2) / (1 + kappa/2) per step, kappa = 2 nu h (1 -
    phi_l)^2 / W0^2."""
    sc, _, _ = _liquid_box(6, 5, undercool=0.3)
    p = sc["params"]
    s = np.full(30, 0.5)
    phi = np.stack([1 - s, s]).reshape(-1)
    mu = np.full(30, 2 * 1.0 * 0.35 * 0.3)
    w, c = oracle.lattice(9)
    f = _feq(w, c, np.ones(30), np.repeat(np.array([[3e-4], [-1e-4]]), 30, axis=1)).reshape(-1)
    _, _, u0 = oracle.derived(sc, phi, mu, f)
    steps = 20
    phi1, _, f1 = oracle.run(sc, phi, mu, f, steps)
    np.testing.assert_array_equal(phi1, phi)
    _, _, u1 = oracle.derived(sc, phi, mu, f1, steps)
    nu = (p["tau_f"] - 0.5) / 3
    kappa = 2 * nu * p["h_drag"] * 0.25 / p["W0"] ** 2
    r = (1 - kappa / 2) / (1 + kappa / 2)
    np.testing.assert_allclose(u1, u0 * r ** steps, rtol=1e-12)


@pytest.mark.parametrize("q", [9, 19, 27])
def test_streaming_moves_population_k_along_c_k(q):
    """tau = 1 makes f* = f^eq; a density excess at one cell then arrives
    one cell along c_k in population k (Eq. LBMEq_1)."""
    dim = 2 if q == 9 else 3
    n = 5
    sc, phi, mu = _liquid_box(n, n, n if dim == 3 else 1, tau_f=1.0)
    sc["grid"]["lattice"] = q
    w, c = oracle.lattice(q)
    cells = n ** dim
    rho = np.ones(cells)
    x0 = (2,) * dim
    idx = np.ravel_multi_index(x0[::-1], (n,) * dim)
    rho[idx] = 1.3
    f = (w[:, None] * rho[None, :]).reshape(-1)
    _, _, f1 = oracle.run(sc, phi, mu, f, 1)
    f1 = f1.reshape(q, cells)
    for k in range(q):
        dest = tuple((np.array(x0) + c[k, :dim]) % n)
        j = np.ravel_multi_index(dest[::-1], (n,) * dim)
        expect = np.full(cells, w[k])
        expect[j] = 1.3 * w[k]
        np.testing.assert_allclose(f1[k], expect, rtol=1e-15)


def _directional(shift, n0=0, V=0.0, steps=300):
    ny = 48
    sc, _, _ = _liquid_box(3, ny, bc=(0, 1, 0), G=4e-3, V=V, v0=20.0)
    p = sc["params"]
    eps = p["eps"]
    yc = p["v0"] + V * n0 + shift
    y = np.arange(ny) + 0.5
    half = math.pi ** 2 * eps / 8
    prof = 0.5 * (1 - np.sin(4 * np.clip(y - yc, -half, half) / (math.pi * eps)))
    s = np.repeat(prof, 3)
    phi = np.stack([1 - s, s]).reshape(-1)
    mu = np.zeros(3 * ny)
    phi1, _, _ = oracle.run(sc, phi, mu, oracle.rest_populations(sc), steps, n0=n0)
    s1 = phi1.reshape(2, ny, 3)[1, :, 1]
    return _crossing(y, prof), _crossing(y, s1)


def test_frozen_temperature_gradient_sets_the_front():
    """T = T_E - u + G (v - v0 - V t): with mu = 0 the front is at rest where
    T = T_E; above it the liquid is stable, so a front placed higher melts
    back and one placed lower grows, and the rest position moves with V t."""
    a, b = _directional(+3.0)
    assert b < a - 0.02
    a, b = _directional(-3.0)
    assert b > a + 0.02
    a, b = _directional(0.0, n0=4000, V=1e-3, steps=100)  # on the moving isotherm
    assert abs(b - a) < 0.02
    a, b = _directional(-4.0, n0=4000, V=1e-3, steps=100)  # at v0: 4 cells below it
    assert b > a + 0.04


def _lamella_pair_rows(v0, steps):
    """Solid rows of one alpha/beta lamella pair of the eutectic2d workload
    (32 x 72, periodic x) after `steps` steps with the isotherm at v0."""
    sc = inputs.scenario("eutectic2d", nx=32, ny=72, precision="fp64")
    sc["params"]["v0"] = v0
    phi, mu = inputs.initial_state(sc)
    oracle.set_threads(oracle.max_threads())
    phi, _, _ = oracle.run(sc, phi, mu, oracle.rest_populations(sc), steps)
    return (1.0 - phi.reshape(3, -1)[0]).sum() / 32.0


def test_eutectic_lamellae_grow_below_their_isotherm():
    """Capillarity of 16-cell lamellae at gamma = 1/5 needs an undercooling of
    about 0.06 to hold them still, far more than G = 1e-4 gives over the grid:
    with T_E at the lamellae's top (v0 = 32) they melt back while the isotherm
    rises; with T_E 0.125 / G above them (the workload's v0) they grow at
    about V = 1e-3 (about 6 rows in 6000 steps)."""
    assert inputs.scenario("eutectic2d")["params"]["v0"] == pytest.approx(1282.0)
    assert _lamella_pair_rows(32.0, 6000) < 32.0 - 1.0
    grown = _lamella_pair_rows(1282.0, 6000)
    assert 32.0 + 2.0 < grown < 32.0 + 20.0


# ----------------------------------------------------------------- moving frame
def _frame_pair(dim, s, n1, n2, lower_v0=True):
    """Window A (nv layers) steps n1 times, moves its frame s layers up the
    material and steps n2 times more; B covers A's first and last windows at
    once (nv + s layers) and steps n1 + n2 times.  A starts from B's seeded
    initial state cut to its first window.  Returns A's final fields and B's,
    the latter cut to A's final window (B layers s .. s + nv)."""
    nv = 84
    if dim == 2:
        big = inputs.scenario("eutectic2d", nx=40, ny=nv + s)
    else:
        big = inputs.scenario("eutectic3d", nx=12, ny=10, nz=nv + s)
        big["init"]["height"] = 32
        big["init"]["noise"] = 1e-3  # seeded, so that the window ends see different values
    big["params"]["G"] = 4e-3  # a strong gradient: a frame without its T shift is visibly off
    big["params"]["v0"] = 32.0 if dim == 2 else 24.0  # isotherm near the solid's top
    phi_b, mu_b = inputs.initial_state(big)
    nx, ny, _ = inputs.dims(big)
    layer = nx * (ny if dim == 3 else 1)
    NP, NC = big["n_phases"], big["n_solutes"]
    small = copy.deepcopy(big)
    small["grid"]["nz" if dim == 3 else "ny"] = nv
    cut = lambda a, k: a.reshape(k, -1)[:, :nv * layer].reshape(-1)
    phi_a, mu_a = cut(phi_b, NP), cut(mu_b, NC)
    f_a, f_b = oracle.rest_populations(small), oracle.rest_populations(big)
    phi_a, mu_a, f_a = oracle.run(small, phi_a, mu_a, f_a, n1)
    phi_a, mu_a, f_a = oracle.shift_frame(small, phi_a, mu_a, f_a, s)
    if lower_v0:
        small["params"]["v0"] -= s
    phi_a, mu_a, f_a = oracle.run(small, phi_a, mu_a, f_a, n2, n0=n1)
    phi_b, mu_b, f_b = oracle.run(big, phi_b, mu_b, f_b, n1 + n2)
    win = lambda a, k: a.reshape(k, -1)[:, s * layer:(s + nv) * layer]
    Q = 19 if dim == 3 else 9
    A = [x.reshape(k, -1) for x, k in ((phi_a, NP), (mu_a, NC), (f_a, Q))]
    B = [win(phi_b, NP), win(mu_b, NC), win(f_b, Q)]
    return A, B, layer


@pytest.mark.parametrize("dim", [2, 3])
def test_moving_frame_matches_the_taller_domain_away_from_its_ends(dim):
    """Moving the window and lowering v0 by the same s changes nothing where
    neither window's ends can be felt: a step reaches at most 2 cells (phi^{n+1}
    of the neighbours enters mu^{n+1}), so layers more than 2 (n1 + n2) + 1
    below A's first top and 2 n2 + 1 above its last bottom agree with the
    taller run to rounding (T = T_E - u + G (v - (v0 - s) - V t) is the same
    number up to the order of its sums)."""
    s, n1, n2 = 10, 6, 6
    A, B, layer = _frame_pair(dim, s, n1, n2)
    lo = 2 * n2 + 1
    hi = 84 - s - 2 * (n1 + n2) - 1
    assert hi - lo >= 20
    band = slice(lo * layer, hi * layer)
    for a, b in zip(A, B):
        np.testing.assert_allclose(a[:, band], b[:, band], rtol=0, atol=1e-12)
    # the ends of the window do differ (the band is not trivially everything)
    assert max(np.abs(a - b).max() for a, b in zip(A, B)) > 1e-9
    # without lowering v0 the frozen temperature slides with the window
    A2, B2, _ = _frame_pair(dim, s, n1, n2, lower_v0=False)
    assert np.abs(A2[0][:, band] - B2[0][:, band]).max() > 1e-7


def test_moving_frame_rejects_bad_shifts():
    sc = inputs.scenario("eutectic2d", nx=8, ny=12)
    phi, mu = inputs.initial_state(sc)
    f = oracle.rest_populations(sc)
    for rows in (-1, 12):
        with pytest.raises(ValueError):
            oracle.shift_frame(sc, phi, mu, f, rows)
    sc["grid"]["wall_rows"] = [0, 2, 0]
    with pytest.raises(ValueError):
        oracle.shift_frame(sc, phi, mu, f, 1)


# ----------------------------------------------------------------- shrinkage
@pytest.mark.parametrize("dim", [2, 3])
def test_shrinkage_momentum_balances_the_solidified_volume(dim):
    """Eq. shrinkage, one step from rest, planar front normal to x between
    walls, no drag (h = 0) and no buoyancy: Guo forcing adds exactly sum_x F
    to the total momentum, and F = F_S, whose x-sum is eta times the solid
    gained with the sign of the normal (the solid lies at low x, so the
    liquid is pulled towards it, -x).  Nothing moves across x = const."""
    if dim == 2:
        sc = inputs.scenario("dendrite2d", nx=40, ny=6)
        sc["grid"]["bc"] = [inputs.WALL, inputs.PERIODIC, inputs.PERIODIC]
        sc["grid"]["wall_rows"] = [0, 0, 0]
    else:
        sc = inputs.scenario("dendrite3d", nx=40, ny=5, nz=4)
        sc["grid"]["bc"] = [inputs.WALL, inputs.PERIODIC, inputs.PERIODIC]
    pr = sc["params"]
    pr["h_drag"] = 0.0
    pr["gbeta_c"] = [0.0, 0.0]
    pr["gbeta_T"] = 0.0
    eta = 0.2
    pr["eta_rho"] = [0.0, eta, 0.0, 0.0]
    nx, ny, nz = inputs.dims(sc)
    x = np.tile(np.arange(nx), ny * nz)
    s = inputs._seed_profile(x + 0.5, 14.0, pr["eps"])  # solid for x < 14
    phi = np.concatenate([1.0 - s, s])
    mu = np.zeros(nx * ny * nz)
    f0 = oracle.rest_populations(sc)
    phi1, mu1, f1 = oracle.run(sc, phi, mu, f0, 1)
    w, c = oracle.lattice(19 if dim == 3 else 9)
    Q, cells = len(w), nx * ny * nz
    f1 = f1.reshape(Q, cells)
    mom = np.array([(c[:, a][:, None] * f1).sum() for a in range(3)])
    grown = phi1[cells:].sum() - s.sum()
    assert grown > 1e-3  # the undercooled front advances
    assert mom[0] == pytest.approx(-eta * grown, rel=1e-10)
    assert abs(mom[1]) < 1e-13 and abs(mom[2]) < 1e-13
    # eta = 0 leaves the fluid at rest
    pr["eta_rho"] = [0.0] * 4
    _, _, f2 = oracle.run(sc, phi, mu, f0, 1)
    assert np.abs(f2 - f0).max() < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_3d_shear_wave_decays_at_the_bgk_viscosity(q):
    """u_x = U sin(k z) in a periodic 3D liquid box decays as exp(-nu k^2 t),
    nu = (tau - 1/2)/3, to second order in k, on D3Q19 and D3Q27."""
    def rate(n, tau=0.8, U=1e-4, t0=20, t1=220):
        sc, phi, mu = _liquid_box(4, 4, n, tau_f=tau)
        sc["grid"]["lattice"] = q
        w, c = oracle.lattice(q)
        cells = 16 * n
        k = 2 * math.pi / n
        z = np.repeat(np.arange(n), 16)
        u = np.zeros((3, cells))
        u[0] = U * np.sin(k * (z + 0.5))
        cu = c.astype(float) @ u
        f = (w[:, None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (u * u).sum(0)[None, :])).reshape(-1)
        amps = []
        for tt in (t0, t1):
            _, _, ff = oracle.run(sc, phi, mu, f, tt)
            _, _, uu = oracle.derived(sc, phi, mu, ff, tt)
            ux = uu.reshape(3, cells)[0]
            amps.append((ux * np.sin(k * (z + 0.5))).sum())
        nu = (tau - 0.5) / 3
        return -math.log(amps[1] / amps[0]) / (t1 - t0) / (nu * k * k)
    r16, r32 = rate(16), rate(32)
    assert abs(r32 - 1) < 3e-3
    assert abs(r16 - 1) / abs(r32 - 1) > 3.0  # second order in k


# ----------------------------------------------------------------- flop counter
def test_flop_counter_is_per_cell_and_per_step():
    """The instrumented oracle (the same steps on a counting number type):
    on a uniform liquid box every cell does the same work, so the count per
    cell-update does not depend on the grid size or the number of steps, and
    the stages add up to the total."""
    counts = []
    for n, steps in ((8, 1), (16, 1), (16, 3)):
        sc, phi, mu = _liquid_box(n, n, bc=(0, 0, 0))
        f = oracle.rest_populations(sc)
        d = oracle.count_flops(sc, phi, mu, f, steps)
        parts = d["phase_field"] + d["macroscopic"] + d["chemical_potential"] + d["lattice_boltzmann"]
        assert d["total"] == pytest.approx(parts, rel=1e-15)
        counts.append(d)
    for d in counts[1:]:
        for k in d:
            assert d[k] == pytest.approx(counts[0][k], rel=1e-15), k
    assert counts[0]["lattice_boltzmann"] > 100 and counts[0]["phase_field"] > 0


# ----------------------------------------------------------------- simplex projection
def _projection_by_enumeration(v):
    """Euclidean projection onto {sum u = 1, u >= 0} by brute force: for every
    support S, the closest point of the affine set {sum_S u = 1, u = 0 off S}
    is u_S = v_S - (sum v_S - 1)/|S|; the projection is the nearest feasible
    one of these (the projection lies on one of these faces)."""
    import itertools
    m = len(v)
    best, best_d = None, np.inf
    for r in range(1, m + 1):
        for S in itertools.combinations(range(m), r):
            u = np.zeros(m)
            idx = list(S)
            u[idx] = v[idx] - (v[idx].sum() - 1.0) / r
            if (u >= -1e-15).all():
                d = ((u - v) ** 2).sum()
                if d < best_d - 1e-15:
                    best, best_d = u, d
    return best


def test_simplex_projection_matches_enumeration_of_supports():
    """The oracle's sort-and-threshold projection [R11] equals the projection
    found by enumerating supports, on random vectors of 1..4 values and on the
    special cases a phase-field update meets (already on the simplex, a tie,
    one large value, all values equal, all negative)."""
    rng = np.random.default_rng(7)
    cases = [np.array(c, dtype=float) for c in (
        [1.0], [0.3], [0.5, 0.5], [1.2, -0.2], [0.2, 0.3, 0.5], [0.4, 0.4, 0.4],
        [2.0, 0.0, 0.0, 0.0], [-0.1, -0.2, -0.3, -0.4], [0.6, 0.6, -0.1, 0.0],
        [0.25, 0.25, 0.25, 0.25], [1.0 + 1e-9, 0.0, -1e-9])]
    for m in (2, 3, 4):
        cases += [rng.normal(1.0 / m, 0.4, m) for _ in range(200)]
    for v in cases:
        got = oracle.project_simplex(v)
        want = _projection_by_enumeration(v)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-14, err_msg=str(v))
        assert abs(got.sum() - 1.0) < 1e-14 and (got >= 0).all()


# ----------------------------------------------------------------- antitrapping
def test_antitrapping_current_cancels_the_thin_interface_trapping():
    """Slow planar front pulled at V through a gradient (tests/thin_interface.py):
    the chemical-potential jump across the interface, normalised by
    2 A v dc eps / D, is -(pi^2/16 - a_at) + O(v eps / D) by the thin-interface
    solute balance of the obstacle profile.  Without the current the jump is
    the trapping level -pi^2/16 at every width; the current adds exactly
    a_at (at a_at = pi^2/16 and pi/4); at a_at = pi^2/16 what is left is
    small and falls with the Peclet number.  A wrong sign, a dropped liquid
    weight, a wrong power of eps or a missing normal in the current fails."""
    import concurrent.futures
    import multiprocessing

    import thin_interface

    a_star = math.pi ** 2 / 16.0
    runs = {("4", "0"): (4.0, 0.0, {}), ("4", "a*"): (4.0, a_star, {}),
            ("8", "0"): (8.0, 0.0, {}), ("8", "a*"): (8.0, a_star, {}),
            ("8", "pi/4"): (8.0, math.pi / 4.0, {}),
            ("8", "a*", "slow"): (8.0, a_star, {"V": 5e-4, "steps": 48000, "L": 300})}
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=min(len(runs), os.cpu_count() or 1),
                                                mp_context=ctx) as pool:
        fut = {k: pool.submit(thin_interface.case, e, a, **kw) for k, (e, a, kw) in runs.items()}
        r = {k: f.result() for k, f in fut.items()}
    for e in ("4", "8"):
        j0, js = r[e, "0"]["jhat"], r[e, "a*"]["jhat"]
        assert r[e, "0"]["jump"] < 0.0                         # the solid traps solute
        assert abs(j0 + a_star) < 0.1, (e, j0)                 # trapping level -pi^2/16
        tol = 0.08 if e == "4" else 0.05
        assert abs((js - j0) / a_star - 1.0) < tol, (e, js - j0)  # the current adds a_at
        assert abs(js) < 0.1 and abs(js) < abs(j0) / 5.0, (e, js)
    jp = r["8", "pi/4"]["jhat"] - r["8", "0"]["jhat"]
    assert abs(jp / (math.pi / 4.0) - 1.0) < 0.05, jp
    assert r["8", "pi/4"]["jhat"] > 0.05                       # pi/4 over-corrects
    slow, fast = r["8", "a*", "slow"], r["8", "a*"]
    assert slow["p"] < 0.6 * fast["p"]
    assert abs(slow["jhat"]) < 0.7 * abs(fast["jhat"]), (slow["jhat"], fast["jhat"])


# ----------------------------------------------------------------- anisotropic faces
def _manufactured_divergence(dim, n, delta, theta):
    """Relative max error of the oracle's discrete divergence of dA/dq at the
    faces, scaled by n^2, against the analytic div(dA/dq(grad S)) for a
    smooth field S without critical points (sampled s(x) = S(x / n), walls
    on every axis, cells at least three from a wall)."""
    sp = pytest.importorskip("sympy")
    q = sp.symbols("q0:%d" % dim, real=True)
    c, s_ = sp.cos(theta), sp.sin(theta)
    r = [c * q[0] + s_ * q[1], -s_ * q[0] + c * q[1]] + ([q[2]] if dim == 3 else [])
    s2 = sum(v ** 2 for v in r)
    s4 = sum(v ** 4 for v in r)
    A = (1 - delta * (3 - 4 * s4 / s2 ** 2)) ** 2 * s2
    hess_A = sp.lambdify(q, sp.hessian(A, q), "numpy")
    X = sp.symbols("X0:%d" % dim, real=True)
    nv = np.array([1.0, 0.7, 0.4][:dim])
    nv /= np.linalg.norm(nv)
    amp = sp.Rational(1, 50) if dim == 2 else sp.Rational(1, 125)
    wave = sp.sin(2 * sp.pi * X[0]) * sp.cos(2 * sp.pi * X[1])
    if dim == 3:
        wave *= sp.sin(2 * sp.pi * X[2])
    S = sp.Rational(1, 2) + sp.Rational(3, 20) * sum(float(nv[i]) * (X[i] - sp.Rational(1, 2))
                                                     for i in range(dim)) + amp * wave
    S_f = sp.lambdify(X, S, "numpy")
    grad_f = [sp.lambdify(X, sp.diff(S, x), "numpy") for x in X]
    hess_f = [[sp.lambdify(X, sp.diff(S, a, b), "numpy") for b in X] for a in X]

    sc = inputs.scenario("dendrite3d" if dim == 3 else "dendrite2d", nx=n, ny=n,
                         nz=n if dim == 3 else None, precision="fp64")
    sc["grid"]["bc"] = [1, 1, 1]
    sc["grid"]["wall_rows"] = [0, 0, 0]
    p = sc["params"]
    p["gbeta_c"], p["gbeta_T"], p["undercool"], p["G"] = [0.0, 0.0], 0.0, 0.0, 0.0
    p["tau_phi"] = 50.0  # a small step: no value leaves (0, 1)
    for a, b in ((0, 1), (1, 0)):
        p["delta"][a][b] = delta
        p["tilt"][a][b] = theta
    idx = np.indices((n,) * dim)[::-1]  # x, y(, z), x fastest
    Xs = [i.reshape(-1) / n for i in idx]
    one = np.ones(n ** dim)
    s0 = S_f(*Xs) * one
    phi1, _, _ = oracle.run(sc, np.concatenate([1.0 - s0, s0]), np.zeros(n ** dim),
                            oracle.rest_populations(sc), 1)
    s1 = phi1[n ** dim:]
    eps, gam, tau = p["eps"], p["gamma"][0][1], p["tau_phi"]
    # N = 2 at mu = 0, T = T_E: tau eps ds/dt = (eps gam Dh - 16 gam (1 - 2 s) / (pi^2 eps)) / 2,
    # Dh the discrete divergence of dA/dq at the faces (centre terms cancel)
    Dh = (2.0 * tau * eps * (s1 - s0) + 16.0 * gam / (math.pi ** 2 * eps) * (1.0 - 2.0 * s0)) / (eps * gam)
    g = [gf(*Xs) * one for gf in grad_f]
    HA = np.array(hess_A(*g), dtype=np.float64)
    div = sum(HA[a][b] * (hess_f[a][b](*Xs) * one) for a in range(dim) for b in range(dim))
    inner = np.all([(i >= 3) & (i <= n - 4) for i in idx], axis=0).reshape(-1)
    return np.abs(n * n * Dh - div)[inner].max() / np.abs(div[inner]).max()


@pytest.mark.parametrize("dim,sizes", [(2, (32, 64, 128)), (3, (16, 32, 64))])
def test_anisotropic_face_divergence_converges_at_second_order(dim, sizes):
    """Manufactured solution for the face stencil [R9] with strong cubic
    anisotropy (delta = 0.3) on turned axes (theta = 0.3): the anisotropic
    flux's normal component depends on the transverse face gradients, so a
    wrong transverse stencil (even one that keeps the cubic symmetry) stops
    the convergence; the error falls four-fold per halving of the spacing."""
    e = [_manufactured_divergence(dim, n, 0.3, 0.3) for n in sizes]
    assert e[-1] < 0.01, e
    assert e[-2] / e[-1] > 3.5 and e[0] / e[1] > 3.0, e


# ----------------------------------------------------------------- objective
def test_objective_of_a_sharp_step_has_the_closed_form():
    """J = w_frac mean h_1 + w_tip tip / nx [R23].  For a sharp solid block the
    mean of h_1 is the solid share of the cells, and along the ray the logits
    are kappa r for r <= R and 0 beyond, so the soft-argmax is a ratio of
    geometric sums: with x = e^kappa and M = nx - 1 - x0,
    tip = [x (1 - (R+1) x^R + R x^(R+1)) / (1-x)^2 + (M(M+1) - R(R+1)) / 2]
          / [(x^(R+1) - 1) / (x - 1) + M - R].
    kappa = 0 gives the plain mean M / 2."""
    nx, ny, x0, y0, R = 48, 20, 10, 9, 13
    sc = inputs.scenario("dendrite2d", nx=nx, ny=ny, precision="fp64")
    solid = np.zeros((ny, nx))
    solid[4:15, 3:x0 + R + 1] = 1.0
    phi = np.concatenate([(1.0 - solid).reshape(-1), solid.reshape(-1)])
    M = nx - 1 - x0
    for kappa in (2.0, 0.7):
        x = math.exp(kappa)
        num = x * (1 - (R + 1) * x ** R + R * x ** (R + 1)) / (1 - x) ** 2 + (M * (M + 1) - R * (R + 1)) / 2
        den = (x ** (R + 1) - 1) / (x - 1) + M - R
        for wf, wt in ((1.0, 0.0), (0.0, 1.0), (0.3, 2.0)):
            obj = {"w_frac": wf, "w_tip": wt, "kappa": kappa, "x0": x0, "y0": y0, "solid": 1}
            J = oracle.objective_value(sc, obj, phi)
            want = wf * solid.sum() / solid.size + wt * (num / den) / nx
            assert J == pytest.approx(want, rel=1e-13, abs=1e-15)
    obj = {"w_frac": 0.0, "w_tip": 1.0, "kappa": 0.0, "x0": x0, "y0": y0, "solid": 1}
    assert oracle.objective_value(sc, obj, phi) == pytest.approx(M / 2.0 / nx, rel=1e-14)


def test_state_tangent_matches_central_differences():
    """The oracle's Jacobian-vector product of the whole state (phi, mu, f
    tangents, forward-mode duals) against central differences of its plain
    steps on a small dendrite with flow, in a direction that keeps the
    phase values away from the clamp."""
    sc = inputs.scenario("dendrite2d", nx=24, ny=20, precision="fp64")
    sc["params"]["gbeta_c"] = [2e-3, 0.0]
    phi0, mu0 = inputs.initial_state(sc)
    w, _ = oracle.lattice(9)
    cells = 24 * 20
    rng = np.random.default_rng(9)
    f0 = (w[:, None] * (1.0 + 1e-3 * rng.normal(size=(9, cells)))).reshape(-1)
    s = phi0.reshape(2, cells)[1]
    ds = rng.normal(size=cells) * ((s > 0.05) & (s < 0.95))
    dphi = np.concatenate([-ds, ds])
    dmu, df = rng.normal(size=cells), 1e-3 * rng.normal(size=9 * cells)
    tp, tm, tf = oracle.tangent(sc, phi0, mu0, f0, 2, dphi=dphi, dmu=dmu, df=df)
    h = 1e-6
    a = oracle.run(sc, phi0 + h * dphi, mu0 + h * dmu, f0 + h * df, 2)
    b = oracle.run(sc, phi0 - h * dphi, mu0 - h * dmu, f0 - h * df, 2)
    for got, pa, pb in zip((tp, tm, tf), a, b):
        fd = (pa - pb) / (2 * h)
        assert np.abs(got - fd).max() <= 1e-6 * max(np.abs(fd).max(), 1e-12)

"""Thin-interface check of the oracle's antitrapping current (test helper).

A planar solid-liquid front of the binary alloy (two phases, one solute,
equal parabolic curvatures A, partition difference dc = ceq_l - ceq_s) is
pulled through a frozen temperature gradient G at speed V on a one-cell-thin
strip, the window following it (moving frame).  Once the front moves
steadily at v, the solute balance across the diffuse interface fixes how
far the chemical potential of the liquid, extrapolated from outside the
interface to the phi = 1/2 point, sits from that of the solid formed there:

    mu_liquid(0) - mu_solid = -(2 A v dc / D) * (I - a_at * eps) + O(p^2),

with p = v eps / D and, for the mobility M = D phi_l / (2 A) and the
interpolation h_l = phi_l^2 (3 - 2 phi_l) on the obstacle profile
phi_l = (1 + sin(4 xi / (pi eps))) / 2,

    I = int (h_l / phi_l - Theta(xi)) dxi = eps * (pi / 4) * (3 pi / 4 - pi / 2) = pi^2 eps / 16,

while the antitrapping current -a_at eps phi_l [c_l - c_s] (dphi_s/dt) n_s,
divided by the same mobility, integrates across the interface to exactly
a_at eps (its phi_l weight cancels the one in M).  The jump normalised by
2 A v dc eps / D is therefore -(pi^2/16 - a_at) + O(p): -pi^2/16 without the
current (solute trapping of order V eps / D), zero at a_at = pi^2/16.

G is set above V / D (the liquidus slope across the boundary layer) so that
the melt ahead of the front is not constitutionally undercooled: otherwise
the diffuse tail of the obstacle profile grows into it.

Each case runs in its own process (spawn), single-threaded.
"""
import math

import numpy as np


def case(eps, a_at, V=1e-3, D=0.1, steps=24000, L=260, y_front=40, c_inf=0.2):
    from oracle import oracle
    from paper_2608_26908_gb300 import inputs

    oracle.set_threads(1)
    nx = 3
    sc = inputs.scenario("dendrite2d", nx=nx, ny=L, precision="fp64")
    sc["grid"]["wall_rows"] = [0, 0, 0]
    p = sc["params"]
    p["eps"], p["W0"], p["a_at"], p["D_liq"] = eps, eps, a_at, D
    p["gbeta_c"], p["gbeta_T"] = [0.0, 0.0], 0.0
    A = p["A"][0]
    dc = p["ceq"][0][0] - p["ceq"][1][0]
    # steady planar front: the solid forms at c_inf, mu = 2 A (c_inf - ceq_s),
    # which rests at the undercooling u = mu / (2 A dc)
    mu_int = 2.0 * A * (c_inf - p["ceq"][1][0])
    G = 1.2 * V / D
    p["undercool"], p["G"], p["V"] = 0.0, G, V
    p["v0"] = y_front + mu_int / (2.0 * A * dc) / G
    y = np.arange(L, dtype=np.float64)
    half = math.pi ** 2 * eps / 8.0
    s = 0.5 * (1.0 - np.sin(4.0 * np.clip(y - y_front, -half, half) / (math.pi * eps)))
    c_liq = c_inf + dc * np.exp(-V * (y - y_front) / D)  # sharp-interface boundary layer
    mu1 = np.where(y < y_front, mu_int, 2.0 * A * (c_liq - p["ceq"][0][0]))
    phi = np.stack([1.0 - s, s])[:, :, None].repeat(nx, axis=2).reshape(-1)
    mu = mu1[:, None].repeat(nx, axis=1).reshape(-1)
    f = oracle.rest_populations(sc)

    def front(ph):
        col = ph.reshape(2, L, nx)[1, :, 0]
        i = np.where((col[:-1] >= 0.5) & (col[1:] < 0.5))[0][0]
        return i + (col[i] - 0.5) / (col[i] - col[i + 1])

    every = int(round(1.0 / V))
    t, shifted, track = 0, 0, []
    while t < steps:
        phi, mu, f = oracle.run(sc, phi, mu, f, every, n0=t)
        t += every
        phi, mu, f = oracle.shift_frame(sc, phi, mu, f, 1)
        sc["params"]["v0"] -= 1.0
        shifted += 1
        track.append((t, front(phi) + shifted))
    (t0, z0), (t1, z1) = track[-4], track[-1]
    v = (z1 - z0) / (t1 - t0)
    col = phi.reshape(2, L, nx)[1, :, 0]
    m = mu.reshape(L, nx)[:, 0]
    yf = front(phi)
    mu_solid = m[np.where(col == 1.0)[0].max()]  # the solid edge of the interface
    first_liquid = np.where(col == 0.0)[0].min()
    ys = np.arange(first_liquid + 1, first_liquid + 1 + int(3 * eps))
    mu_liquid0 = np.polyval(np.polyfit(ys - yf, m[ys], 2), 0.0)
    jump = mu_liquid0 - mu_solid
    return {"eps": eps, "a_at": a_at, "V": V, "v": v, "p": v * eps / D, "jump": jump,
            "jhat": jump / (2.0 * A * v * dc * eps / D)}

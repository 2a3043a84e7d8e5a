"""Brute force on tiny grids: one full time step computed node by node with
plain Python loops, organised differently from the oracle, must agree with
the oracle to 1e-13.

Differences of organisation (so that a slip in one is not repeated in the
other): the velocity set is rebuilt from its definition; neighbours are
found by explicit index arithmetic; the filter is applied as the explicit
Q x Q matrix of the footnote to Eq. 12 (F_ij = Phi_i : c_j c_j) acting on the
non-equilibrium vector; streaming is done by pushing each post-collision
population to its destination instead of pulling.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import lattice as L
from oracle import pflbm as O
from paper_1812_00118_gb300 import inputs as I

T = 1.0 / 3.0


def velocity_set(dim):
    if dim == 2:
        cs = [(a, b, 0) for a, b in itertools.product((-1, 0, 1), repeat=2)]
        wt = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}
    else:
        cs = [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in v) <= 2]
        wt = {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}
    return cs, [wt[sum(x * x for x in c)] for c in cs]


def brute_step(h, g, cs, ws, n, prm, walls):
    """h, g: dict (node, velocity) -> value.  n = (nx, ny, nz).  walls[a] True if axis a is walled."""
    nx, ny, nz = n
    Q = len(cs)
    nodes = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]

    def nb(node, c):                       # phi ghost behind a wall = adjacent node
        out = []
        for a in range(3):
            v = node[a] + c[a]
            if walls[a]:
                v = min(max(v, 0), n[a] - 1)
            else:
                v %= n[a]
            out.append(v)
        return tuple(out)

    phi = {x: sum(h[(x, c)] for c in cs) for x in nodes}
    filt = [[ws[i] / (2 * T * T) * (sum(cs[i][a] * cs[i][b] * cs[j][a] * cs[j][b]
                                         for a in range(3) for b in range(3))
                                     - T * sum(cs[j][a] ** 2 for a in range(3)))
             for j in range(Q)] for i in range(Q)]
    rho_dif = prm["rho_H"] - prm["rho_L"]
    tau_phi = prm["M"] / T + 0.5
    tL = prm["nu_L"] / T + 0.5
    tH = prm["nu_H"] / T + 0.5
    hs, gs = {}, {}
    for x in nodes:
        f = phi[x]
        grad = [0.0, 0.0, 0.0]
        lap = 0.0
        for c, w in zip(cs, ws):
            up, dn = phi[nb(x, c)], phi[nb(x, tuple(-v for v in c))]
            for a in range(3):
                grad[a] += (up - dn) * c[a] * w / (2 * T)
            lap += 2 * (up - f) * w / T
        rho = prm["rho_L"] + f * rho_dif
        mu = 48 * prm["sigma"] / prm["W"] * f * (f - 1) * (f - 0.5) - 1.5 * prm["sigma"] * prm["W"] * lap
        F = [rho * ga for ga in prm["g"]]
        J = [sum(c[a] * g[(x, c)] for c in cs) + 0.5 * (mu * grad[a] + F[a]) for a in range(3)]
        rho_e = rho + 0.25 * rho_dif * lap
        u = [J[a] / rho_e for a in range(3)]
        ug = sum(u[a] * grad[a] for a in range(3))
        P = T * sum(g[(x, c)] for c in cs) + 0.5 * T * rho_dif * ug
        gnorm = math.sqrt(sum(v * v for v in grad))
        nrm = [v / (gnorm + 1e-10) for v in grad]
        th = prm["M"] / T * (1 - 4 * (f - 0.5) ** 2) / prm["W"]
        usq = sum(v * v for v in u)
        pc = min(max(f, 0.0), 1.0)
        om = 1 / tL + pc * (1 / tH - 1 / tL)
        geq, K = [], []
        for c, w in zip(cs, ws):
            cu = sum(c[a] * u[a] for a in range(3))
            Gam = w * (1 + cu / T + cu * cu / (2 * T * T) - usq / (2 * T))
            heq = f * Gam + th * w * sum(c[a] * nrm[a] for a in range(3))
            hs[(x, c)] = h[(x, c)] - (h[(x, c)] - heq) / tau_phi
            k = ((Gam - w) * rho_dif + Gam * mu / T) * sum((c[a] - u[a]) * grad[a] for a in range(3)) \
                + Gam * sum((c[a] - u[a]) * F[a] for a in range(3)) / T
            K.append(k)
            geq.append(rho * Gam + w * (P / T - rho) - 0.5 * k + w * cu * rho_dif * lap / (4 * T))
        neq = [g[(x, c)] - geq[j] for j, c in enumerate(cs)]
        for i, c in enumerate(cs):
            gs[(x, c)] = geq[i] + K[i] + (1 - om) * sum(filt[i][j] * neq[j] for j in range(Q))
    # push streaming with halfway bounce-back
    hn, gn = {}, {}
    for x in nodes:
        for c in cs:
            dest = []
            blocked = False
            for a in range(3):
                v = x[a] + c[a]
                if walls[a] and (v < 0 or v >= n[a]):
                    blocked = True
                dest.append(v % n[a])
            back = tuple(-v for v in c)
            if blocked:
                hn[(x, back)] = hs[(x, c)]
                gn[(x, back)] = gs[(x, c)]
            else:
                hn[(tuple(dest), c)] = hs[(x, c)]
                gn[(tuple(dest), c)] = gs[(x, c)]
    return hn, gn


@pytest.mark.parametrize("lat,n", [(L.D2Q9, (4, 3, 1)), (L.D3Q19, (3, 4, 3))], ids=["D2Q9", "D3Q19"])
@pytest.mark.parametrize("walls", [(False, False, False), (False, True, False), (True, False, True)],
                         ids=["periodic", "ywall", "xzwall"])
def test_single_step_brute_force(lat, n, walls):
    if lat.dim == 2 and walls[2]:
        walls = (walls[0], walls[1], False)
    nx, ny, nz = n
    shape = (nz, ny, nx)
    phi, u, P = I.smooth_random(shape, 31, dim=lat.dim, u_amp=0.03)
    g_acc = (1e-4, -2e-4, 3e-4 if lat.dim == 3 else 0.0)
    prm = dict(M=0.1, W=3.0, sigma=0.02, rho_L=0.001, rho_H=1.0, nu_L=0.1, nu_H=0.02, g=g_acc)
    bc = tuple("wall" if w else "periodic" for w in walls)
    p = O.Params(bc=bc, **prm)
    h, g = O.init_populations(phi, u, P, lat, p)
    rng = np.random.default_rng(32)
    h = h + rng.normal(scale=1e-3, size=h.shape)
    g = g + rng.normal(scale=1e-4, size=g.shape)
    h1, g1 = O.step(h, g, lat, p)

    cs, ws = velocity_set(lat.dim)
    index = {tuple(int(v) for v in lat.c[i]): i for i in range(lat.Q)}
    nodes = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
    hd = {(x, c): h[index[c], x[2], x[1], x[0]] for x in nodes for c in cs}
    gd = {(x, c): g[index[c], x[2], x[1], x[0]] for x in nodes for c in cs}
    hb, gb = brute_step(hd, gd, cs, ws, n, prm, walls)
    for x in nodes:
        for c in cs:
            assert hb[(x, c)] == pytest.approx(h1[index[c], x[2], x[1], x[0]], abs=1e-13)
            assert gb[(x, c)] == pytest.approx(g1[index[c], x[2], x[1], x[0]], abs=1e-13)

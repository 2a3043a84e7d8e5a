"""Seeded synthetic inputs (phi, u, P) shaped like the paper's test cases.

This module holds no arithmetic of the LB method: it only builds initial
fields.  Both the GPU library's tests and the oracle's tests take their
inputs from here; neither side imports the other.

Fields are numpy float64 arrays in (nz, ny, nx) order (x fastest); a 2-D
field is (1, ny, nx).  Velocities are (3, nz, ny, nx).

Recipes (the paper publishes no dataset; these stand in for its cases):

* ``sphere``: a drop (phi = 1 inside) or bubble (phi = 0 inside) of radius
  R with the flat-interface profile phi = 1/2 + 1/2 tanh(2 d / W) across the
  interface (Section 4.1 static droplet; d the signed distance), u = 0,
  P = 0.
* ``layers``: two fluid layers split normal to an axis (Section 3 Poiseuille
  and Couette set-ups), tanh interfaces.
* ``smooth_random``: a periodic field of a few random Fourier modes, phi in
  [0.05, 0.95], small random u and P, for brute-force and parity tests on
  tiny grids with a ragged tail.
* ``batch_cases``: the list of independent D2Q9 drop/bubble cases of uneven
  size for the batched launch.
"""
import numpy as np


def sphere(shape, centre, R, W, drop=True, periodic=True):
    """(phi, u, P) for a static drop or bubble; shape = (nz, ny, nx)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d2 = np.zeros(shape)
    for coord, n, c0 in ((x, nx, centre[0]), (y, ny, centre[1]), (z, nz, centre[2])):
        if n == 1:
            continue
        dd = coord - c0
        if periodic:
            dd = (dd + n / 2.0) % n - n / 2.0
        d2 += dd * dd
    r = np.sqrt(d2)
    s = 1.0 if drop else -1.0
    phi = 0.5 + 0.5 * np.tanh(s * 2.0 * (R - r) / W)
    return phi, np.zeros((3,) + shape), np.zeros(shape)


def layers(shape, axis, split, W, heavy_low=True):
    """(phi, u, P): heavy fluid (phi = 1) below coordinate ``split`` along
    ``axis`` (0 = x, 1 = y, 2 = z), light fluid above, one tanh interface."""
    nz, ny, nx = shape
    coord = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")[2 - axis]
    s = 1.0 if heavy_low else -1.0
    phi = 0.5 + 0.5 * np.tanh(s * 2.0 * (split - coord) / W)
    return phi, np.zeros((3,) + shape), np.zeros(shape)


def smooth_random(shape, seed, modes=3, u_amp=0.02, P_amp=1e-3, dim=3):
    """Random smooth periodic (phi, u, P).  phi in [0.05, 0.95]."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def field():
        f = np.zeros(shape)
        for _ in range(modes):
            kx = rng.integers(0, 3) * 2 * np.pi / nx
            ky = rng.integers(0, 3) * 2 * np.pi / ny
            kz = rng.integers(0, 3) * 2 * np.pi / nz if nz > 1 else 0.0
            f += rng.uniform(-1, 1) * np.cos(kx * x + ky * y + kz * z + rng.uniform(0, 2 * np.pi))
        f += 0.1 * rng.uniform(-1, 1, size=shape)
        m = np.abs(f).max()
        return f / m if m > 0 else f

    phi = 0.5 + 0.45 * field()
    u = np.zeros((3,) + shape)
    for a in range(dim):
        u[a] = u_amp * field()
    P = P_amp * field()
    return phi, u, P


def batch_cases(n_cases=512, L_min=32, L_max=512, seed=0):
    """Independent D2Q9 static drop/bubble cases of uneven size.

    Square sides L uniform on the integers [L_min, L_max]; R = L/4 +- U(0, L/16);
    density ratio log-uniform in [10, 1000] (rho_H = 1); tau uniform in
    [0.51, 0.8] for both phases; W in {3, 4, 5}; drop or bubble 50/50.  Each
    case draws from its own generator seeded with (seed, index)."""
    cases = []
    for k in range(n_cases):
        rng = np.random.default_rng([seed, k])
        L = int(rng.integers(L_min, L_max + 1))
        R = L / 4.0 + rng.uniform(-1.0, 1.0) * rng.uniform(0.0, L / 16.0)
        ratio = float(np.exp(rng.uniform(np.log(10.0), np.log(1000.0))))
        tau = float(rng.uniform(0.51, 0.8))
        W = float(rng.choice([3.0, 4.0, 5.0]))
        drop = bool(rng.integers(0, 2))
        cases.append(dict(L=L, R=R, rho_ratio=ratio, tau=tau, W=W, drop=drop))
    return cases


def drops(L, seed, n_min=1, n_max=4, R_min=12.0, R_max=48.0, W=4.0, gap=None, bubbles=False):
    """(phi, u, P, drops) of 1-4 static drops (phi = 1 inside) in a periodic
    L x L box, shape (1, L, L): radii uniform in [R_min, R_max], centres
    uniform and off the nodes, drops at least `gap` (default 2 W) apart along
    the periodic distance, phi the sum of the tanh profiles (clipped to 1).
    With `bubbles` the phases are exchanged: light-phase bubbles (phi = 0
    inside) in the heavy phase.  A drop that finds no room after 200 tries is
    left out; the drop list gives (x, y, R)."""
    rng = np.random.default_rng([seed, 1812])
    gap = 2.0 * W if gap is None else gap
    n = int(rng.integers(n_min, n_max + 1))
    placed = []
    for _ in range(n):
        for _attempt in range(200):
            R = float(rng.uniform(R_min, min(R_max, L / 2.0 - W)))
            c = rng.uniform(0.0, L, size=2) + 0.31
            ok = True
            for (px, py, pR) in placed:
                d = np.abs(np.array([c[0] - px, c[1] - py]))
                d = np.minimum(d, L - d)
                if np.hypot(*d) < R + pR + gap:
                    ok = False
                    break
            if ok:
                placed.append((float(c[0]), float(c[1]), R))
                break
    if not placed:
        placed.append((L / 2.0 + 0.31, L / 2.0 - 0.23, R_min))
    phi = np.zeros((1, L, L))
    for (cx, cy, R) in placed:
        p, _, _ = sphere((1, L, L), (cx, cy, 0.0), R, W, drop=True)
        phi += p
    phi = np.minimum(phi, 1.0)
    if bubbles:
        phi = 1.0 - phi
    return phi, np.zeros((3, 1, L, L)), np.zeros((1, L, L)), placed


def perturbed_interface(nx, ny, W, amplitude=0.1):
    """(ny, nx) phi of a flat horizontal interface at ny / 2 with a cosine
    perturbation of one wavelength nx and amplitude `amplitude` * nx, heavy
    fluid (phi = 1) above: the Rayleigh-Taylor start of Section 4 (the paper
    gives no perturbation; this one is a reading)."""
    Y, X = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    y0 = ny / 2 + amplitude * nx * np.cos(2 * np.pi * (X + 0.5) / nx)
    return 0.5 + 0.5 * np.tanh(2 * (Y - y0) / W)

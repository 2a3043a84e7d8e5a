"""Validation diagnostics of the oracle (Section 4.1, the static droplet).

The paper measures the pressure jump dP across a static droplet and checks
Laplace's law dP = sigma / R in two dimensions.  It does not say where P is
sampled; the reading here is: dP = <P>_{r < R - 2W} - <P>_{r > R + 2W}
(distances with periodic wrap), and the effective radius comes from the
order parameter: R = sqrt(V / pi) in 2-D, (3 V / (4 pi))^(1/3) in 3-D,
V = sum phi for a drop, sum (1 - phi) for a bubble.  In 3-D the law is
dP = 2 sigma / R.
"""
import numpy as np


def radial_distance(shape, centre, periodic=True):
    """|x - centre| for a (nz, ny, nx) grid, minimum-image if periodic."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = []
    for coord, n, c0 in ((x, nx, centre[0]), (y, ny, centre[1]), (z, nz, centre[2])):
        dd = coord - c0
        if periodic:
            dd = (dd + n / 2.0) % n - n / 2.0
        d.append(dd)
    return np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)


def laplace_jump(P, centre, R, W, drop=True, periodic=True):
    """dP = P_inside - P_outside, sampled away from the interface."""
    r = radial_distance(P.shape, centre, periodic)
    inside = P[r < R - 2.0 * W].mean()
    outside = P[r > R + 2.0 * W].mean()
    return float(inside - outside)


def effective_radius(phi, dim, drop=True):
    V = float(phi.sum()) if drop else float((1.0 - phi).sum())
    if dim == 2:
        return np.sqrt(V / np.pi)
    return (3.0 * V / (4.0 * np.pi)) ** (1.0 / 3.0)


def totals(phi, rho):
    """Global sum of phi and of mass (conserved under periodic boundaries)."""
    return float(phi.sum()), float(rho.sum())


def rt_fronts(phi, nx, ny):
    """Rayleigh-Taylor fronts (Section 4) in units of the width L = nx,
    measured from the initial interface height ny / 2: the lowest row
    holding heavy fluid (phi > 1/2, the spike tip, negative) and the highest
    row holding light fluid (the bubble tip, positive)."""
    heavy = np.asarray(phi).reshape(ny, nx) > 0.5
    spike = np.where(heavy.any(axis=1))[0].min()
    bubble = np.where((~heavy).any(axis=1))[0].max()
    return (spike - ny / 2) / nx, (bubble - ny / 2) / nx

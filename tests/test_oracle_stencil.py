"""Pins of the central-difference stencils (unnumbered equations after Eq. 12).

Closed forms: the stencils are exact for linear (gradient) and quadratic
(Laplacian) fields away from boundaries, and on a periodic sine mode along
an axis they reduce to the textbook symbols sin(k) and -4 sin^2(k/2), the
same for D2Q9 and D3Q19 because sum over c_x != 0 of w_i equals T.
"""
import numpy as np
import pytest

from oracle import lattice as L
from oracle import pflbm as O

WALLS = ("wall", "wall", "wall")


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19], ids=lambda l: l.name)
def test_linear_and_quadratic_exactness(lat):
    shape = (7, 8, 9) if lat.dim == 3 else (1, 8, 9)
    z, y, x = np.meshgrid(*[np.arange(s, dtype=float) for s in shape], indexing="ij")
    inner = (slice(1, -1) if lat.dim == 3 else slice(None), slice(1, -1), slice(1, -1))
    a = np.array([0.3, -0.7, 1.1 if lat.dim == 3 else 0.0])
    lin = a[0] * x + a[1] * y + a[2] * z + 0.25
    gr = O.gradient(lin, lat, WALLS)
    for k in range(3):
        np.testing.assert_allclose(gr[k][inner], a[k], atol=1e-14)
    np.testing.assert_allclose(O.laplacian(lin, lat, WALLS)[inner], 0.0, atol=1e-14)
    quad = x * x + 2 * y * y - x * y + (3 * z * z if lat.dim == 3 else 0.0)
    lap_exact = 2 + 4 + (6 if lat.dim == 3 else 0)
    np.testing.assert_allclose(O.laplacian(quad, lat, WALLS)[inner], lap_exact, atol=1e-12)
    gq = O.gradient(quad, lat, WALLS)
    np.testing.assert_allclose(gq[0][inner], (2 * x - y)[inner], atol=1e-12)
    np.testing.assert_allclose(gq[1][inner], (4 * y - x)[inner], atol=1e-12)


AXIS_CASES = [(L.D2Q9, 0), (L.D2Q9, 1), (L.D3Q19, 0), (L.D3Q19, 1), (L.D3Q19, 2)]
AXIS_IDS = ["D2Q9-x", "D2Q9-y", "D3Q19-x", "D3Q19-y", "D3Q19-z"]


@pytest.mark.parametrize("lat,axis", AXIS_CASES, ids=AXIS_IDS)
def test_fourier_symbols(lat, axis):
    n = 16
    shape = [1, 1, 1]
    shape[2 - axis] = n
    k = 2 * np.pi * 3 / n
    s = np.arange(n)
    phi = np.sin(k * s).reshape(shape)
    bc = ("periodic",) * 3
    gr = O.gradient(phi, lat, bc)[axis].reshape(-1)
    np.testing.assert_allclose(gr, np.sin(k) * np.cos(k * s), atol=1e-14)
    lap = O.laplacian(phi, lat, bc).reshape(-1)
    np.testing.assert_allclose(lap, -4 * np.sin(k / 2) ** 2 * np.sin(k * s), atol=1e-14)


@pytest.mark.parametrize("lat,axis", AXIS_CASES, ids=AXIS_IDS)
def test_wall_nodes_read_the_adjacent_fluid_value(lat, axis):
    """Reading R9: behind a wall the stencils read the value of the fluid
    node next to it (zero normal gradient).  For phi = a s along a walled
    axis s the central difference at the first node is then (phi(1) -
    phi(0)) / 2 = a/2 and the Laplacian phi(1) - phi(0) = a (the weights of
    the directions with c_s = +1 sum to 1/6 on both lattices, so the
    stencils reduce to the 1-D differences); at the last node a/2 and -a."""
    shape = (6, 7, 8) if lat.dim == 3 else (1, 7, 8)
    coords = np.meshgrid(*[np.arange(s, dtype=float) for s in shape], indexing="ij")
    s = coords[2 - axis]
    a = 0.37
    phi = a * s + 0.1
    gr = O.gradient(phi, lat, WALLS)
    lap = O.laplacian(phi, lat, WALLS)
    first = [slice(None)] * 3
    last = [slice(None)] * 3
    first[2 - axis], last[2 - axis] = 0, -1
    np.testing.assert_allclose(gr[axis][tuple(first)], a / 2, atol=1e-14)
    np.testing.assert_allclose(gr[axis][tuple(last)], a / 2, atol=1e-14)
    np.testing.assert_allclose(lap[tuple(first)], a, atol=1e-13)
    np.testing.assert_allclose(lap[tuple(last)], -a, atol=1e-13)
    for b in range(3):
        if b != axis:
            np.testing.assert_allclose(gr[b], 0.0, atol=1e-14)

"""Closed-form pins of the oracle's validation diagnostics (Section 4.1):
the effective radius from the phi volume, the Laplace jump sampled away
from the interface, and the minimum-image distance they use."""
import numpy as np
import pytest

from oracle import diagnostics as D
from paper_1812_00118_gb300 import inputs as I


@pytest.mark.parametrize("dim,R,drop", [(2, 14.3, True), (2, 11.7, False), (3, 9.6, True), (3, 8.2, False)])
def test_effective_radius_of_a_tanh_sphere(dim, R, drop):
    """V of 0.5 + 0.5 tanh(2 (R - r) / W) is the ball of radius R up to the
    O((W / R)^2) relative term of the profile's curvature: pi R^2 (1 +
    pi^2 W^2 / (48 R^2)) in 2-D, 4/3 pi R^3 (1 + pi^2 W^2 / (16 R^2)) in 3-D
    (the Sommerfeld expansion of the Fermi-like profile).  A bubble measures
    the light-phase volume."""
    W = 2.0
    shape = (1, 48, 48) if dim == 2 else (32, 32, 32)
    nz, ny, nx = shape
    centre = ((nx - 1) / 2 + 0.31, (ny - 1) / 2 - 0.17, (nz - 1) / 2 + 0.23 if dim == 3 else 0.0)
    phi = I.sphere(shape, centre, R, W, drop=drop)[0]
    corr = (np.pi ** 2 * W * W / (48.0 * R * R)) if dim == 2 else (np.pi ** 2 * W * W / (16.0 * R * R))
    R_exact = R * (1.0 + corr) ** (1.0 / dim)
    assert D.effective_radius(phi, dim, drop) == pytest.approx(R_exact, rel=2e-3)
    # the other dimension's formula or the other phase is far off
    assert abs(D.effective_radius(phi, 5 - dim, drop) - R_exact) > 0.05 * R
    assert abs(D.effective_radius(phi, dim, not drop) - R_exact) > 0.5 * R


def test_laplace_jump_of_a_step_field():
    """P = a inside r < R, b outside: the jump is a - b whatever the band
    excluded around the interface, and it changes sign with the fields."""
    shape = (20, 22, 24)
    centre = (11.4, 10.6, 9.8)
    r = D.radial_distance(shape, centre)
    P = np.where(r < 7.0, 0.3, -0.05)
    assert D.laplace_jump(P, centre, 7.0, 1.0) == pytest.approx(0.35, abs=1e-15)
    assert D.laplace_jump(-P, centre, 7.0, 1.5) == pytest.approx(-0.35, abs=1e-15)


def test_radial_distance_minimum_image():
    shape = (1, 10, 12)
    d = D.radial_distance(shape, (0.0, 0.0, 0.0))
    assert d[0, 0, 11] == pytest.approx(1.0)           # wraps to the neighbour of x = 0
    assert d[0, 9, 0] == pytest.approx(1.0)
    assert d[0, 5, 6] == pytest.approx(np.hypot(5.0, 6.0))
    dn = D.radial_distance(shape, (0.0, 0.0, 0.0), periodic=False)
    assert dn[0, 0, 11] == pytest.approx(11.0)

"""Pins of the diffusion correction of Eq. 14 (Section 3) in the oracle.

The paper leaves the function F of delta theta = C (M/T) F |grad phi| open;
the oracle's reading R18 takes F = -W^2 max(0, (2 phi - 1) lap phi).  What the
mathematics fixes, checked here:

* C = 0 is the model of Section 2, bit for bit;
* F vanishes on the tanh profile of Eq. 4 (continuum: (2 phi - 1) phi'' <= 0)
  and on its nodal samples with the CD stencil, at any offset and width;
* delta theta enters h^eq only through theta w_i (c_i . n): sum_i h^eq_i = phi
  is kept and the first moment becomes phi u + (theta + delta theta) T n;
* on an ordinary bubble it stays two orders below theta, so its evolution
  barely changes;
* on a dense bubble (a shallow dip of phi inside the heavy phase, where
  (2 phi - 1) lap phi > 0) it adds diffusion: the dip the Allen-Cahn model
  sharpens ends shallower with C > 0 than with C = 0.
"""
import numpy as np
import pytest

from oracle import lattice as L
from oracle import pflbm as O
from paper_1812_00118_gb300 import inputs as I

T = L.T


def test_zero_constant_is_section_2_model():
    phi, u, P = I.smooth_random((6, 7, 8), 3)
    a = O.Params(M=0.1, W=3.0)
    b = O.Params(M=0.1, W=3.0, C_dtheta=0.0)
    ha, ga = O.init_populations(phi, u, P, L.D3Q19, a)
    hb, gb = O.init_populations(phi, u, P, L.D3Q19, b)
    ha, ga = O.run(ha, ga, L.D3Q19, a, 3)
    hb, gb = O.run(hb, gb, L.D3Q19, b, 3)
    assert np.array_equal(ha, hb) and np.array_equal(ga, gb)


@pytest.mark.parametrize("W,offset", [(2.5, 0.0), (3.0, 0.3), (4.0, 0.5), (5.0, 0.77)])
def test_vanishes_on_tanh_profile(W, offset):
    """F = 0 at every node of a flat tanh interface sampled on the lattice,
    both orientations (heavy phase on either side)."""
    n = 64
    for heavy_low in (True, False):
        phi, u, P = I.layers((1, 1, n), axis=0, split=n / 2 - 0.5 + offset, W=W, heavy_low=heavy_low)
        p = O.Params(M=0.1, W=W, C_dtheta=3.0, bc=("wall", "periodic", "periodic"))
        grad = O.gradient(phi, L.D2Q9, p.bc)
        lap = O.laplacian(phi, L.D2Q9, p.bc)
        dth = O.delta_theta(phi, grad, lap, p)
        assert np.abs(dth).max() == 0.0


def test_continuum_sign_on_tanh():
    """(2 phi - 1) phi'' <= 0 on phi = 1/2 + 1/2 tanh(2x/W), with phi'' from
    its closed form (16/W^2) phi (1 - phi)(1 - 2 phi)."""
    x = np.linspace(-20, 20, 4001)
    for W in (2.5, 4.0):
        phi = 0.5 + 0.5 * np.tanh(2 * x / W)
        d2 = np.gradient(np.gradient(phi, x), x)
        closed = (16 / W ** 2) * phi * (1 - phi) * (1 - 2 * phi)
        assert np.abs(d2 - closed).max() < 1e-3 * np.abs(closed).max()
        assert ((2 * phi - 1) * closed).max() <= 0.0


def test_moments_with_correction():
    """sum_i h^eq_i = phi; sum_i c_i h^eq_i = phi u + (theta + delta theta) T n."""
    phi, u, P = I.smooth_random((7, 8, 9), 12)
    p = O.Params(M=0.13, W=3.0, C_dtheta=2.0)
    lat = L.D3Q19
    grad = O.gradient(phi, lat, p.bc)
    lap = O.laplacian(phi, lat, p.bc)
    heq = O.h_equilibrium(phi, u, grad, lat, p, lap=lap)
    dth = O.delta_theta(phi, grad, lap, p)
    assert np.abs(dth).max() > 1e-3 * np.abs(O.theta(phi, p)).max()   # the case exercises it
    np.testing.assert_allclose(heq.sum(axis=0), phi, atol=1e-14)
    n = O.normal(grad, p)
    first = np.einsum("ia,i...->a...", lat.c.astype(float), heq)
    expect = phi[None] * u + ((O.theta(phi, p) + dth) * T)[None] * n
    np.testing.assert_allclose(first, expect, atol=1e-14)
    # and the correction is exactly what separates it from C = 0
    p0 = O.Params(M=0.13, W=3.0)
    heq0 = O.h_equilibrium(phi, u, grad, lat, p0)
    first0 = np.einsum("ia,i...->a...", lat.c.astype(float), heq0)
    np.testing.assert_allclose(first - first0, (dth * T)[None] * n, atol=1e-14)


def test_small_on_ordinary_bubble():
    n = 48
    phi, u, P = I.sphere((1, n, n), (23.6, 24.3, 0), 12.0, 3.0, drop=False)
    p = O.Params(M=0.17, W=3.0, C_dtheta=1.0)
    grad = O.gradient(phi, L.D2Q9, p.bc)
    lap = O.laplacian(phi, L.D2Q9, p.bc)
    ratio = np.abs(O.delta_theta(phi, grad, lap, p)).max() / O.theta(phi, p).max()
    assert ratio < 1e-2, ratio


@pytest.mark.slow
def test_dense_bubble_is_diffused():
    """A shallow dip (phi_min = 0.92) inside the heavy phase: the Allen-Cahn
    counter-term deepens it into a dense bubble; with C = 5 the dip ends at
    most two thirds as deep, while an ordinary bubble of radius 12 moves by
    less than 3e-2 in phi."""
    n = 48
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r2 = (x - 23.6) ** 2 + (y - 24.3) ** 2
    dip = (1.0 - 0.08 * np.exp(-r2 / 18.0))[None]
    z3 = np.zeros((3, 1, n, n))
    z1 = np.zeros((1, n, n))
    depth = {}
    for C in (0.0, 5.0):
        p = O.Params(M=0.17, W=3.0, sigma=0.01, rho_L=1e-3, rho_H=1.0, nu_L=0.17, nu_H=0.17, C_dtheta=C)
        h, g = O.init_populations(dip, z3, z1, L.D2Q9, p)
        h, g = O.run(h, g, L.D2Q9, p, 1000)
        depth[C] = 1.0 - h.sum(axis=0).min()
    assert depth[0.0] > 0.2                      # the model of Section 2 nucleates it
    assert depth[5.0] < (2.0 / 3.0) * depth[0.0], depth
    phi, u, P = I.sphere((1, n, n), (23.6, 24.3, 0), 12.0, 3.0, drop=False)
    out = {}
    for C in (0.0, 5.0):
        p = O.Params(M=0.17, W=3.0, sigma=0.01, rho_L=1e-3, rho_H=1.0, nu_L=0.17, nu_H=0.17, C_dtheta=C)
        h, g = O.init_populations(phi, u, P, L.D2Q9, p)
        h, g = O.run(h, g, L.D2Q9, p, 1000)
        out[C] = h.sum(axis=0)
    assert np.abs(out[5.0] - out[0.0]).max() < 3e-2

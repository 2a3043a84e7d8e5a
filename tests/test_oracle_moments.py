"""Closed-form pins of the oracle's local operators (Section 2, Eqs. 2-13).

Each test checks a moment identity that follows from the paper's
definitions plus lattice isotropy, computed independently of the oracle's
per-direction loops (einsum over the velocity table here).  A dropped term,
a wrong sign or a transposed index in h^eq, K_i, g^eq, delta f^eq, the
Hermite filter or the recovery formulas breaks at least one of them.
"""
import numpy as np
import pytest

from oracle import lattice as L
from oracle import pflbm as O
from paper_1812_00118_gb300 import inputs as I

T = 1.0 / 3.0
LATS = [L.D2Q9, L.D3Q19]


def mom0(f):
    return f.sum(axis=0)


def mom1(f, lat):
    return np.einsum("ia,i...->a...", lat.c.astype(float), f)


def mom2(f, lat):
    c = lat.c.astype(float)
    return np.einsum("ia,ib,i...->ab...", c, c, f)


def random_local_state(lat, seed, shape=(3, 4, 5)):
    """Random independent node values (no spatial structure needed here)."""
    rng = np.random.default_rng(seed)
    if lat.dim == 2:
        shape = (1,) + shape[1:]
    phi = rng.uniform(-0.05, 1.05, shape)
    u = np.zeros((3,) + shape)
    u[: lat.dim] = rng.uniform(-0.05, 0.05, (lat.dim,) + shape)
    grad = np.zeros((3,) + shape)
    grad[: lat.dim] = rng.uniform(-0.3, 0.3, (lat.dim,) + shape)
    lap = rng.uniform(-0.2, 0.2, shape)
    P = rng.uniform(-1e-3, 1e-3, shape)
    return phi, u, grad, lap, P


def params(lat, **kw):
    g = (1e-4, -2e-4, 3e-4) if lat.dim == 3 else (1e-4, -2e-4, 0.0)
    base = dict(M=0.1, W=4.0, sigma=0.01, rho_L=0.001, rho_H=1.0, nu_L=0.05, nu_H=0.01, g=g)
    base.update(kw)
    return O.Params(**base)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_gamma_moments(lat):
    phi, u, grad, lap, P = random_local_state(lat, 1)
    G = O.gamma(u, lat)
    np.testing.assert_allclose(mom0(G), 1.0, atol=1e-15)
    np.testing.assert_allclose(mom1(G, lat), u, atol=1e-16)
    I3 = np.eye(3)[:, :, None, None, None]
    if lat.dim == 2:
        I3 = np.diag([1.0, 1.0, 0.0])[:, :, None, None, None]
    np.testing.assert_allclose(mom2(G, lat), T * I3 + np.einsum("a...,b...->ab...", u, u), atol=1e-15)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_h_equilibrium_moments(lat):
    """sum h^eq = phi (phi = sum h must be invariant); first moment phi u + theta T n."""
    p = params(lat)
    phi, u, grad, lap, P = random_local_state(lat, 2)
    heq = O.h_equilibrium(phi, u, grad, lat, p)
    np.testing.assert_allclose(mom0(heq), phi, atol=1e-15)
    mag = np.sqrt((grad ** 2).sum(0))
    n = grad / (mag + p.eps)
    th = (p.M / T) * 4.0 * phi * (1.0 - phi) / p.W        # 1 - 4(phi - 1/2)^2 = 4 phi (1 - phi)
    np.testing.assert_allclose(mom1(heq, lat), phi * u + T * th * n, atol=1e-15)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_forcing_moments(lat):
    """K_i carries the force: sum K = rho_dif u.grad phi, sum c K = mu grad phi + F,
    and the second moment has the closed form of the third moments of Gamma."""
    p = params(lat)
    phi, u, grad, lap, P = random_local_state(lat, 3)
    rho = O.density(phi, p)
    mu = O.chemical_potential(phi, lap, p)
    F = O.external_force(rho, p)
    K = O.forcing(u, grad, mu, F, lat, p)
    ug = (u * grad).sum(0)
    uF = (u * F).sum(0)
    np.testing.assert_allclose(mom0(K), p.rho_dif * ug, atol=1e-15)
    np.testing.assert_allclose(mom1(K, lat), mu * grad + F, atol=1e-15)
    s = p.rho_dif + mu / T
    d = lat.dim
    Id = np.diag([1.0] * d + [0.0] * (3 - d))[:, :, None, None, None]
    outer = lambda a, b: np.einsum("a...,b...->ab...", a, b)
    expect = s * (T * (outer(u, grad) + outer(grad, u)) - outer(u, u) * ug) \
        + p.rho_dif * T * Id * ug \
        + (T * (outer(u, F) + outer(F, u)) - outer(u, u) * uF) / T
    np.testing.assert_allclose(mom2(K, lat), expect, atol=1e-14)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
@pytest.mark.parametrize("hocorr", [True, False])
def test_g_equilibrium_moments(lat, hocorr):
    """The recovery formulas after Eq. 12 invert g^eq: sum g^eq = P/T - rho_dif u.grad phi/2,
    sum c g^eq = (rho + lap rho / 4) u - (mu grad phi + F)/2 (reading R4)."""
    p = params(lat, hocorr=hocorr)
    phi, u, grad, lap, P = random_local_state(lat, 4)
    rho = O.density(phi, p)
    mu = O.chemical_potential(phi, lap, p)
    F = O.external_force(rho, p)
    K = O.forcing(u, grad, mu, F, lat, p)
    geq = O.g_equilibrium(rho, u, P, K, lap, lat, p)
    ug = (u * grad).sum(0)
    np.testing.assert_allclose(mom0(geq), P / T - 0.5 * p.rho_dif * ug, atol=1e-14)
    rho_eff = rho + (0.25 * p.rho_dif * lap if hocorr else 0.0)
    np.testing.assert_allclose(mom1(geq, lat), rho_eff * u - 0.5 * (mu * grad + F), atol=1e-15)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_high_order_correction_moments(lat):
    """Eq. 13 has zero mass, first moment u lap(rho)/4 and zero second moment."""
    p = params(lat)
    phi, u, grad, lap, P = random_local_state(lat, 5)
    d = O.high_order_correction(u, lap, lat, p)
    np.testing.assert_allclose(mom0(d), 0.0, atol=1e-17)
    np.testing.assert_allclose(mom1(d, lat), 0.25 * p.rho_dif * lap * u, atol=1e-17)
    np.testing.assert_allclose(mom2(d, lat), 0.0, atol=1e-17)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_hermite_filter(lat):
    """Phi_i : Pi (Eq. 11) has no mass, no momentum and second moment Pi."""
    rng = np.random.default_rng(6)
    shape = (2, 3, 4)
    A = rng.normal(size=(3, 3) + shape)
    A = A + A.transpose(1, 0, 2, 3, 4)
    if lat.dim == 2:
        A[2, :] = 0.0
        A[:, 2] = 0.0
    proj = O.hermite_projection(A, lat)
    np.testing.assert_allclose(mom0(proj), 0.0, atol=1e-14)
    np.testing.assert_allclose(mom1(proj, lat), 0.0, atol=1e-14)
    np.testing.assert_allclose(mom2(proj, lat), A, atol=1e-13)


def test_chemical_potential_vanishes_on_flat_profile():
    """For phi = 1/2 + 1/2 tanh(2x/W) the two terms of Eq. 8 cancel exactly in
    the continuum; with the exact second derivative the oracle gives mu = 0.
    The same profile makes theta T / M equal to |phi'| (Eq. 4)."""
    p = O.Params(sigma=0.013, W=3.7, M=0.07)
    x = np.linspace(-10, 10, 401)
    s = np.tanh(2 * x / p.W)
    phi = 0.5 + 0.5 * s
    dphi = (1 - s * s) / p.W
    d2phi = -(4.0 / p.W ** 2) * s * (1 - s * s)
    mu = O.chemical_potential(phi, d2phi, p)
    assert np.abs(mu).max() < 1e-15
    th = O.theta(phi, p)
    np.testing.assert_allclose(th * T / p.M, dphi, atol=1e-15)
    # surface tension: (3 sigma W / 2) int phi'^2 dx = sigma
    assert 1.5 * p.sigma * p.W * np.trapezoid(dphi ** 2, x) == pytest.approx(p.sigma, rel=1e-6)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
@pytest.mark.parametrize("force_mode", [0, 1])
def test_init_macro_roundtrip(lat, force_mode):
    """Initialising with the equilibria and recovering (phi, u, P) by the formulas
    after Eq. 12 returns the input to round-off."""
    shape = (5, 6, 7) if lat.dim == 3 else (1, 9, 11)
    phi, u, P = I.smooth_random(shape, 7, dim=lat.dim)
    p = params(lat, force_mode=force_mode)
    h, g = O.init_populations(phi, u, P, lat, p)
    m = O.macroscopic(h, g, lat, p)
    np.testing.assert_allclose(m["phi"], phi, atol=1e-15)
    np.testing.assert_allclose(m["u"], u, atol=1e-16)
    np.testing.assert_allclose(m["P"], P, atol=1e-16)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_collision_moments(lat):
    """Per node: h collision keeps phi; g collision adds rho_dif u.grad phi to the
    mass moment and mu grad phi + F to the momentum moment (Eqs. 5-7, R4);
    the post-collision non-equilibrium lies in the second-order Hermite space."""
    shape = (5, 6, 7) if lat.dim == 3 else (1, 9, 11)
    phi, u, P = I.smooth_random(shape, 8, dim=lat.dim)
    p = params(lat)
    h, g = O.init_populations(phi, u, P, lat, p)
    # push the state off equilibrium with a random perturbation that keeps the
    # conserved moments of h (sum) and g (sum and first moment)
    rng = np.random.default_rng(9)
    dh = rng.normal(scale=1e-3, size=h.shape)
    dh -= dh.mean(axis=0)
    h = h + dh
    g = g + O.hermite_projection(_sym(rng, shape, lat), lat) + _third_order_noise(rng, lat, shape)
    m = O.macroscopic(h, g, lat, p)
    hs, gs = O.collide(h, g, lat, p, m)
    np.testing.assert_allclose(mom0(hs), mom0(h), atol=1e-15)
    ug = (m["u"] * m["grad"]).sum(0)
    np.testing.assert_allclose(mom0(gs) - mom0(g), p.rho_dif * ug, atol=1e-14)
    np.testing.assert_allclose(mom1(gs, lat) - mom1(g, lat), m["mu"] * m["grad"] + m["F"], atol=1e-14)
    G = O.gamma(m["u"], lat)
    K = O.forcing(m["u"], m["grad"], m["mu"], m["F"], lat, p, G)
    geq = O.g_equilibrium(m["rho"], m["u"], m["P"], K, m["lap"], lat, p, G)
    neq = gs - geq - K
    np.testing.assert_allclose(O.hermite_projection(mom2(neq, lat), lat), neq, atol=1e-14)


def _sym(rng, shape, lat):
    A = rng.normal(scale=1e-4, size=(3, 3) + shape)
    A = A + A.transpose(1, 0, 2, 3, 4)
    if lat.dim == 2:
        A[2, :] = 0.0
        A[:, 2] = 0.0
    return A


def _third_order_noise(rng, lat, shape):
    """A perturbation with zero mass, momentum and second moment (higher-order
    content only), which the filter must remove."""
    c = lat.c.astype(float)
    basis = np.concatenate([np.ones((1, lat.Q)), c.T, np.einsum("ia,ib->abi", c, c).reshape(9, lat.Q)])
    r = rng.normal(scale=1e-4, size=(lat.Q,) + shape).reshape(lat.Q, -1)
    # remove the component in the span of the low-order moment rows
    U, sv, _ = np.linalg.svd(basis.T, full_matrices=False)
    Qm = U[:, sv > 1e-10]
    r = r - Qm @ (Qm.T @ r)
    return r.reshape((lat.Q,) + shape)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_filtered_equals_bgk_on_hermite_nonequilibrium(lat):
    """Eq. 10 is Eq. 5 with the non-equilibrium projected on the second-order
    Hermite space, so the two agree exactly when g - g^eq already lies there."""
    shape = (4, 5, 6) if lat.dim == 3 else (1, 7, 8)
    phi, u, P = I.smooth_random(shape, 10, dim=lat.dim)
    p = params(lat)
    h, g = O.init_populations(phi, u, P, lat, p)
    rng = np.random.default_rng(11)
    g = g + O.hermite_projection(_sym(rng, shape, lat), lat)
    pf = params(lat, collision="filtered")
    pb = params(lat, collision="bgk")
    _, gf = O.collide(h, g, lat, pf)
    _, gb = O.collide(h, g, lat, pb)
    np.testing.assert_allclose(gf, gb, atol=1e-15)
    # and they differ when higher-order content is present
    g2 = g + _third_order_noise(rng, lat, shape)
    _, gf2 = O.collide(h, g2, lat, pf)
    _, gb2 = O.collide(h, g2, lat, pb)
    assert np.abs(gf2 - gb2).max() > 1e-6


def test_tau_mix_interpolation():
    """Eq. 9 endpoints: phi = 1 is water (heavy, nu_H), phi = 0 air (nu_L); nu = T (tau - 1/2)."""
    p = O.Params(nu_L=0.17, nu_H=0.0017)
    om = O.inv_tau_mix(np.array([0.0, 1.0, -0.1, 1.1, 0.5]), p)
    assert T * (1 / om[0] - 0.5) == pytest.approx(0.17, rel=1e-14)
    assert T * (1 / om[1] - 0.5) == pytest.approx(0.0017, rel=1e-14)
    assert om[2] == om[0] and om[3] == om[1]
    assert om[4] == pytest.approx(0.5 * (om[0] + om[1]), rel=1e-15)


def test_chapman_enskog_rebuild():
    """Reading R19: g = g^eq + Phi : Pi(1) keeps the zeroth and first moments
    of g^eq (so the rebuilt state has the given P and u), its non-equilibrium
    second moment is Pi(1) itself, and on a sheared single-phase flow that has
    relaxed under the filtered collision the measured pre-collision
    non-equilibrium momentum flux agrees with Pi(1) = -tau T rho (du + du^T)."""
    from oracle import lattice as LL
    from paper_1812_00118_gb300 import inputs as II
    lat = LL.D3Q19
    phi, u, P = II.smooth_random((6, 7, 8), 21)
    p = O.Params(M=0.1, W=4.0, sigma=0.01, rho_L=0.1, rho_H=1.0, nu_L=0.05, nu_H=0.02)
    h0, g0 = O.init_populations(phi, u, P, lat, p)
    h1, g1 = O.init_populations(phi, u, P, lat, p, nonequilibrium=True)
    assert np.array_equal(h0, h1)
    d = g1 - g0
    c = lat.c.astype(float)
    np.testing.assert_allclose(d.sum(axis=0), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("ia,i...->a...", c, d), 0.0, atol=1e-16)
    Pi = O.chapman_enskog_pi(phi, u, lat, p)
    np.testing.assert_allclose(O.second_moment(d, lat), Pi, atol=1e-15)
    # single phase (phi = 1), a long shear wave u_x = U sin(k y) decaying under
    # the filtered collision: after it has relaxed onto its slow mode the
    # pre-collision sum c c (g - g^eq) matches Pi(1) to O(k^2)
    ny = 64
    k = 2 * np.pi / ny
    q = O.Params(M=0.1, W=4.0, sigma=0.0, rho_L=1.0, rho_H=1.0, nu_L=0.05, nu_H=0.05, hocorr=False,
                 modified_velocity=False)
    shape = (1, ny, 1)
    phi1 = np.ones(shape)
    uu = np.zeros((3,) + shape)
    uu[0] = 1e-3 * np.sin(k * np.arange(ny))[None, :, None]

    def mismatch(hh, gg):
        m = O.macroscopic(hh, gg, lat, q)
        G = O.gamma(m["u"], lat)
        K = O.forcing(m["u"], m["grad"], m["mu"], m["F"], lat, q, G)
        geq = O.g_equilibrium(m["rho"], m["u"], m["P"], K, m["lap"], lat, q, G)
        meas = O.second_moment(gg - geq, lat)[0, 1]
        est = O.chapman_enskog_pi(m["phi"], m["u"], lat, q)[0, 1]
        return np.abs(meas - est).max() / np.abs(est).max()

    hh, gg = O.init_populations(phi1, uu, np.zeros(shape), lat, q)
    assert mismatch(*O.run(hh, gg, lat, q, 300)) < 0.01      # relaxed: O(k^2) apart (2e-3)
    assert mismatch(*O.run(hh, gg, lat, q, 1)) > 0.3         # an equilibrium start is not
    hn, gn = O.init_populations(phi1, uu, np.zeros(shape), lat, q, nonequilibrium=True)
    assert mismatch(*O.run(hn, gn, lat, q, 1)) < 0.01        # the rebuilt start already is

"""Physics pins of the oracle: what the paper and the continuum limit fix.

* exact global conservation of phi and mass under periodic boundaries and
  under bounce-back walls (Eq. 1 conserves sum_i h_i at every node);
* the momentum bookkeeping of Eqs. 5-7: sum_x sum_i c_i g_i changes per step
  by exactly sum_x (mu grad phi + F);
* diffusion of a sine mode at rate M k^2 (Eq. 1 with tau = M/T + 1/2);
* shear-wave decay at nu k^2 in either pure phase (Eq. 9 endpoints, filter);
* Laplace's law dP = sigma / R for a static drop and bubble at density
  ratio 1000 (Section 4.1), converging as the interface is resolved, and
  dP = 2 sigma / R for a 3-D bubble;
* the layered two-phase Poiseuille profile against FP64 quadrature of
  d/dy(rho nu u') = -rho g with the diffuse interface and mixed viscosity
  (Section 3), and the interface peak of the uncorrected model that Eq. 13
  removes;
* Galilean test of Section 3 (uniformly advected drop keeps its velocity).
"""
import numpy as np
import pytest
from scipy.integrate import cumulative_trapezoid

from oracle import diagnostics as D
from oracle import lattice as L
from oracle import pflbm as O
from paper_1812_00118_gb300 import inputs as I

T = 1.0 / 3.0


@pytest.mark.parametrize("lat,shape", [(L.D2Q9, (1, 13, 17)), (L.D3Q19, (5, 7, 9))],
                         ids=["D2Q9", "D3Q19"])
@pytest.mark.parametrize("walls", [False, True])
def test_global_conservation(lat, shape, walls):
    phi, u, P = I.smooth_random(shape, 21, dim=lat.dim)
    bc = ("periodic", "wall", "periodic") if walls else ("periodic",) * 3
    g_acc = (2e-5, 0.0, 1e-5) if lat.dim == 3 else (2e-5, 0.0, 0.0)
    p = O.Params(M=0.1, W=3.0, sigma=0.01, rho_L=0.01, rho_H=1.0, nu_L=0.1, nu_H=0.05,
                 g=g_acc, bc=bc)
    h, g = O.init_populations(phi, u, P, lat, p)
    phi0 = O.order_parameter(h).sum()
    c = lat.c.astype(float)
    for _ in range(30):
        m = O.macroscopic(h, g, lat, p)
        mom_before = np.einsum("ia,ixyz->a", c, g)
        source = (m["mu"][None] * m["grad"] + m["F"]).reshape(3, -1).sum(axis=1)
        h, g = O.step(h, g, lat, p)
        if not walls:
            mom_after = np.einsum("ia,ixyz->a", c, g)
            np.testing.assert_allclose(mom_after - mom_before, source, atol=1e-14)
    phi1 = O.order_parameter(h).sum()
    assert abs(phi1 - phi0) < 1e-12 * phi0
    rho0 = O.density(phi, p).sum()
    rho1 = O.density(O.order_parameter(h), p).sum()
    assert abs(rho1 - rho0) < 1e-12 * rho0


def _mode_amplitude(f, k, x):
    return 2.0 * np.mean(f * np.sin(k * x))


@pytest.mark.parametrize("lat,shape", [(L.D2Q9, (1, 1, 128)), (L.D3Q19, (128, 1, 1))],
                         ids=["D2Q9-x", "D3Q19-z"])
def test_diffusion_rate_is_mobility(lat, shape):
    """With u = 0, no surface tension and theta -> 0 (W -> inf) Eq. 1 is a
    diffusion equation with diffusivity T (tau_phi - 1/2) = M."""
    p = O.Params(M=0.1, W=1e12, sigma=0.0, rho_L=1.0, rho_H=1.0, nu_L=0.1, nu_H=0.1)
    n = max(shape)
    k = 2 * np.pi / n
    x = np.arange(n)
    phi = (0.5 + 0.1 * np.sin(k * x)).reshape(shape)
    h, g = O.init_populations(phi, np.zeros((3,) + shape), np.zeros(shape), lat, p)
    h, g = O.run(h, g, lat, p, 50)
    a1 = _mode_amplitude(O.order_parameter(h).reshape(-1), k, x)
    h, g = O.run(h, g, lat, p, 400)
    a2 = _mode_amplitude(O.order_parameter(h).reshape(-1), k, x)
    rate = np.log(a1 / a2) / 400
    assert rate == pytest.approx(p.M * k * k, rel=1e-3)


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19], ids=lambda l: l.name)
@pytest.mark.parametrize("phase", [1.0, 0.0], ids=["heavy", "light"])
def test_shear_wave_viscosity(lat, phase):
    """Single phase (phi = 1 or 0): mu = 0, grad phi = 0, and the filtered
    collision (Eq. 10) must give nu = T (tau - 1/2) of that phase (Eq. 9)."""
    p = O.Params(M=0.1, W=4, sigma=0.01, rho_L=0.001, rho_H=1.0, nu_L=0.05, nu_H=0.1)
    shape = (1, 128, 1)
    n = 128
    k = 2 * np.pi / n
    y = np.arange(n)
    phi = np.full(shape, phase)
    u = np.zeros((3,) + shape)
    u[0] = (1e-3 * np.sin(k * y)).reshape(shape)
    h, g = O.init_populations(phi, u, np.zeros(shape), lat, p)

    def amp():
        return _mode_amplitude(O.macroscopic(h, g, lat, p)["u"][0].reshape(-1), k, y)

    h, g = O.run(h, g, lat, p, 50)
    a1 = amp()
    h, g = O.run(h, g, lat, p, 400)
    a2 = amp()
    nu = p.nu_H if phase == 1.0 else p.nu_L
    assert np.log(a1 / a2) / 400 == pytest.approx(nu * k * k, rel=1e-3)


def _laplace(R, W, sigma, steps, nu_H=0.17, mu_ratio=60.0, drop=True):
    """Static drop (or bubble) of Section 4.1: box 5R, periodic, rho ratio
    1000, M = 0.1.  Returns dP / (sigma / R), dP = P inside - P outside."""
    N = int(5 * R)
    p = O.Params(M=0.1, W=W, sigma=sigma, rho_L=1e-3, rho_H=1.0,
                 nu_L=nu_H * 1000.0 / mu_ratio, nu_H=nu_H)
    shape = (1, N, N)
    centre = (N / 2, N / 2, 0)
    phi, u, P = I.sphere(shape, centre, R, W, drop=drop)
    h, g = O.init_populations(phi, u, P, L.D2Q9, p)
    h, g = O.run(h, g, L.D2Q9, p, steps)
    m = O.macroscopic(h, g, L.D2Q9, p)
    Reff = D.effective_radius(m["phi"], 2, drop)
    return D.laplace_jump(m["P"], centre, Reff, W) / (sigma / Reff)


@pytest.mark.slow
def test_laplace_law_2d():
    """dP = sigma/R within 8 % at W = 4 (R/W = 3); the error shrinks as W grows
    from the paper's W = 2.5; dP is linear in sigma."""
    r4 = _laplace(12, 4.0, 0.01, 2500)
    r25 = _laplace(12, 2.5, 0.01, 2500)
    assert abs(r4 - 1) < 0.08
    assert abs(r25 - 1) < 0.2
    assert abs(r4 - 1) < abs(r25 - 1)
    r25b = _laplace(12, 2.5, 0.006, 2500)
    assert r25b == pytest.approx(r25, rel=0.02)


def _laplace_jump(R, W, sigma, steps):
    """(R_eff, dP) of the relaxed static drop of _laplace."""
    N = int(5 * R)
    p = O.Params(M=0.1, W=W, sigma=sigma, rho_L=1e-3, rho_H=1.0, nu_L=0.17 * 1000.0 / 60.0, nu_H=0.17)
    shape = (1, N, N)
    centre = (N / 2, N / 2, 0)
    phi, u, P = I.sphere(shape, centre, R, W)
    h, g = O.init_populations(phi, u, P, L.D2Q9, p)
    h, g = O.run(h, g, L.D2Q9, p, steps)
    m = O.macroscopic(h, g, L.D2Q9, p)
    Reff = D.effective_radius(m["phi"], 2, True)
    return Reff, D.laplace_jump(m["P"], centre, Reff, W)


@pytest.mark.slow
def test_laplace_slope_is_sigma():
    """Section 4.1 plots dP against 1/R for drops of several radii and finds
    the slope equal to sigma: a least-squares line through R = 10, 14, 20
    (W = 4, density ratio 1000) has slope sigma within 5 % and an intercept
    within 5 % of the jumps (measured 0.976 sigma, -2.6 %)."""
    sigma = 0.01
    res = [_laplace_jump(R, 4.0, sigma, 2500) for R in (10, 14, 20)]
    x = np.array([1.0 / r for r, _ in res])
    y = np.array([d for _, d in res])
    slope, icpt = np.linalg.lstsq(np.vstack([x, np.ones_like(x)]).T, y, rcond=None)[0]
    assert slope == pytest.approx(sigma, rel=0.05)
    assert abs(icpt) < 0.05 * y.mean()


@pytest.mark.slow
def test_laplace_law_at_the_papers_low_viscosity():
    """Section 4.1's own parameter set: R = 8, 12, 16 in a periodic box of
    5 R, nu_water = 3.3e-4 (tau = 0.501), viscosity ratio 60, M = 0.1, W =
    2.5, density ratio 1000, sigma = 1e-2 in the paper's units (1e-5 with the
    heavy density 1, reading 16).  So little viscosity leaves the acoustic
    waves of the start almost undamped and the instantaneous jump swings by
    tens of percent, so dP is averaged over steps 1000-4000 (every 10th).
    The averaged jumps follow sigma / R within 20 % (the W = 2.5 surface
    tension error of the 2-D pins; measured 0.88, 0.87, 0.85) and their line
    against 1/R has slope sigma within 15 % (0.90) through the origin
    within 8 % of the jumps (-4 %)."""
    sigma, W, nu_H = 1e-5, 2.5, 3.3e-4
    res = []
    for R in (8, 12, 16):
        N = 5 * R
        p = O.Params(M=0.1, W=W, sigma=sigma, rho_L=1e-3, rho_H=1.0, nu_L=nu_H * 1000.0 / 60.0, nu_H=nu_H)
        shape = (1, N, N)
        centre = (N / 2, N / 2, 0)
        phi, u, P = I.sphere(shape, centre, R, W)
        h, g = O.init_populations(phi, u, P, L.D2Q9, p)
        h, g = O.run(h, g, L.D2Q9, p, 1000)
        jumps = []
        for _ in range(300):
            m = O.macroscopic(h, g, L.D2Q9, p)
            Reff = D.effective_radius(m["phi"], 2, True)
            jumps.append(D.laplace_jump(m["P"], centre, Reff, W))
            h, g = O.run(h, g, L.D2Q9, p, 10)
        dP = float(np.mean(jumps))
        assert abs(dP / (sigma / Reff) - 1.0) < 0.2, (R, dP / (sigma / Reff))
        res.append((Reff, dP))
    x = np.array([1.0 / r for r, _ in res])
    y = np.array([d for _, d in res])
    slope, icpt = np.linalg.lstsq(np.vstack([x, np.ones_like(x)]).T, y, rcond=None)[0]
    assert slope == pytest.approx(sigma, rel=0.15)
    assert abs(icpt) < 0.08 * y.mean()


@pytest.mark.slow
def test_laplace_law_2d_bubble():
    """A light bubble in the heavy phase: the pressure inside is again the
    higher one, by sigma / R (the surface force mu grad(phi) integrates to
    the same jump whichever phase the interface encloses)."""
    r = _laplace(12, 4.0, 0.01, 2500, drop=False)
    assert abs(r - 1) < 0.08


@pytest.mark.slow
def test_laplace_law_3d_bubble():
    """Section 4.1 in three dimensions: a bubble at density ratio 1000 holds
    dP = 2 sigma / R (two principal curvatures), R from the volume of the
    light phase (the 3-D branch of effective_radius).  R = 8, W = 3 in a
    32^3 periodic box, centre off the nodes; the jump is established within
    the 250 steps (sound crosses the box in ~55 steps)."""
    R, W, N, sigma = 8.0, 3.0, 32, 0.01
    p = O.Params(M=0.1, W=W, sigma=sigma, rho_L=1e-3, rho_H=1.0, nu_L=0.17 * 1000.0 / 60.0, nu_H=0.17)
    centre = (N / 2 + 0.31, N / 2 - 0.23, N / 2 + 0.17)
    phi, u, P = I.sphere((N, N, N), centre, R, W, drop=False)
    h, g = O.init_populations(phi, u, P, L.D3Q19, p)
    h, g = O.run(h, g, L.D3Q19, p, 250)
    m = O.macroscopic(h, g, L.D3Q19, p)
    Reff = D.effective_radius(m["phi"], 3, drop=False)
    assert abs(Reff - R) < 0.5
    ratio = D.laplace_jump(m["P"], centre, Reff, W) / (2.0 * sigma / Reff)
    assert abs(ratio - 1) < 0.1
    # the 2-D law would be off by a factor two
    assert abs(ratio - 0.5) > 0.3


def _poiseuille(ratio, hocorr, ny=32, steps=6000, W=2.5):
    """Section 3: water below, air above, walls at y = -1/2 and ny - 1/2,
    body force rho g along x, mu_ratio = 100, nu_water = 0.17, M = 0.1."""
    p = O.Params(M=0.1, W=W, sigma=0.01, rho_L=1.0 / ratio, rho_H=1.0,
                 nu_L=0.17 * ratio / 100.0, nu_H=0.17, g=(1e-6, 0.0, 0.0), force_mode=0,
                 bc=("periodic", "wall", "periodic"), hocorr=hocorr, modified_velocity=hocorr)
    shape = (1, ny, 1)
    phi, u, P = I.layers(shape, axis=1, split=ny / 2 - 0.5, W=W)
    h, g = O.init_populations(phi, u, P, L.D2Q9, p)
    with np.errstate(all="ignore"):
        h, g = O.run(h, g, L.D2Q9, p, steps)
    m = O.macroscopic(h, g, L.D2Q9, p)
    ux = m["u"][0].reshape(-1)
    # analytic: d/dy (eta u') = -rho g, eta = rho T (tau_mix - 1/2), u = 0 at the walls
    y = np.linspace(-0.5, ny - 0.5, 40001)
    phif = 0.5 + 0.5 * np.tanh(2 * ((ny / 2 - 0.5) - y) / W)
    rho = p.rho_L + phif * p.rho_dif
    om = 1 / p.tau_L + phif * (1 / p.tau_H - 1 / p.tau_L)
    eta = rho * T * (1 / om - 0.5)
    S = -cumulative_trapezoid(rho * p.g[0], y, initial=0.0)
    A = cumulative_trapezoid(S / eta, y, initial=0.0)
    B = cumulative_trapezoid(1 / eta, y, initial=0.0)
    ua = A - (A[-1] / B[-1]) * B
    u_nodes = np.interp(np.arange(ny), y, ua)
    return np.abs(ux - u_nodes).max() / np.abs(u_nodes).max()


@pytest.mark.slow
def test_layered_poiseuille():
    err_1000 = _poiseuille(1000.0, True)
    err_100 = _poiseuille(100.0, True)
    err_100_orig = _poiseuille(100.0, False)
    assert err_1000 < 0.04
    assert err_100 < 0.01
    # the model without Eq. 13 shows the interface peak the paper reports
    assert err_100_orig > 0.2


def _galilean(hocorr, steps=2000):
    """Section 3: 1-D periodic L = 100, drop in the centre, u = 0.025 everywhere,
    nu_water = 1.7e-2, W = 3, mu_ratio = 100, M = 0.1."""
    nx, W = 100, 3.0
    p = O.Params(M=0.1, W=W, sigma=0.01, rho_L=1e-3, rho_H=1.0, nu_L=0.17, nu_H=0.017,
                 hocorr=hocorr, modified_velocity=hocorr)
    shape = (1, 1, nx)
    x = np.arange(nx)
    phi = (0.5 + 0.5 * np.tanh(2 * (20 - np.abs(x - 49.5)) / W)).reshape(shape)
    u = np.zeros((3,) + shape)
    u[0] = 0.025
    h, g = O.init_populations(phi, u, np.zeros(shape), L.D2Q9, p)
    with np.errstate(all="ignore"):
        h, g = O.run(h, g, L.D2Q9, p, steps)
    m = O.macroscopic(h, g, L.D2Q9, p)
    dev = np.abs(m["u"][0] - 0.025).max() / 0.025
    return dev if np.isfinite(dev) else np.inf


@pytest.mark.slow
def test_galilean_advection():
    assert _galilean(True) < 0.1
    assert _galilean(False) > 0.5


def test_flat_interface_profile_is_stationary():
    """A flat interface initialised with the tanh profile of Eq. 4's width W
    stays within 2e-2 of it (discretisation error at W = 4) and does not move."""
    W = 4.0
    p = O.Params(M=0.1, W=W, sigma=0.01, rho_L=1e-3, rho_H=1.0, nu_L=0.1, nu_H=0.1,
                 bc=("wall", "periodic", "periodic"))
    shape = (1, 1, 48)
    phi, u, P = I.layers(shape, axis=0, split=23.5, W=W)
    h, g = O.init_populations(phi, u, P, L.D2Q9, p)
    h, g = O.run(h, g, L.D2Q9, p, 3000)
    m = O.macroscopic(h, g, L.D2Q9, p)
    assert np.abs(m["phi"] - phi).max() < 2e-2
    # interface position: the phi = 1/2 crossing stays at 23.5
    f = m["phi"].reshape(-1)
    j = np.where((f[:-1] >= 0.5) & (f[1:] < 0.5))[0][0]
    x_half = j + (f[j] - 0.5) / (f[j] - f[j + 1])
    assert abs(x_half - 23.5) < 0.05
    assert np.abs(m["u"]).max() < 1e-6


# ---------------------------------------------------------------- moving walls (R15)
def _couette(ratio, hocorr, moving, ny=32, steps=6000, W=2.5, U=1e-3):
    """Section 3 Couette flow: water below, air above, walls at y = -1/2 and
    ny - 1/2, one of them sliding along x with U (the water-side or the
    air-side wall), mu_ratio = 100, nu_water = 0.17, M = 0.1.  Returns the
    error against the quadrature of (eta u')' = 0 with the diffuse interface
    and mixed viscosity (normalised by U), and the change of sum phi."""
    wu = [(0.0, 0.0, 0.0)] * 6
    wu[2 + (0 if moving == "water" else 1)] = (U, 0.0, 0.0)
    p = O.Params(M=0.1, W=W, sigma=0.01, rho_L=1.0 / ratio, rho_H=1.0, nu_L=0.17 * ratio / 100.0, nu_H=0.17,
                 bc=("periodic", "wall", "periodic"), hocorr=hocorr, modified_velocity=hocorr, wall_u=tuple(wu))
    shape = (1, ny, 1)
    phi, u, P = I.layers(shape, axis=1, split=ny / 2 - 0.5, W=W)
    h, g = O.init_populations(phi, u, P, L.D2Q9, p)
    with np.errstate(all="ignore"):
        h, g = O.run(h, g, L.D2Q9, p, steps)
    m = O.macroscopic(h, g, L.D2Q9, p)
    ux = m["u"][0].reshape(-1)
    # analytic: eta u' is constant across the channel, u = the wall velocities at the walls
    y = np.linspace(-0.5, ny - 0.5, 40001)
    phif = 0.5 + 0.5 * np.tanh(2 * ((ny / 2 - 0.5) - y) / W)
    rho = p.rho_L + phif * p.rho_dif
    om = 1 / p.tau_L + phif * (1 / p.tau_H - 1 / p.tau_L)
    eta = rho * T * (1 / om - 0.5)
    B = cumulative_trapezoid(1 / eta, y, initial=0.0)
    u0, u1 = (U, 0.0) if moving == "water" else (0.0, U)
    ua = u0 + (u1 - u0) * B / B[-1]
    u_nodes = np.interp(np.arange(ny), y, ua)
    return np.abs(ux - u_nodes).max() / U, abs(m["phi"].sum() - phi.sum())


def test_single_phase_couette_is_linear():
    """A sliding wall over one fluid: the steady profile of halfway walls is
    exactly linear, u = U (y + 1/2) / ny, and phi stays 1."""
    U, ny = 0.01, 16
    wu = ((0.0, 0.0, 0.0),) * 3 + ((U, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 2
    p = O.Params(M=0.1, W=3.0, sigma=0.01, rho_L=1e-3, rho_H=1.0, nu_L=1 / 6, nu_H=1 / 6,
                 bc=("periodic", "wall", "periodic"), wall_u=wu)
    shape = (1, ny, 1)
    h, g = O.init_populations(np.ones(shape), np.zeros((3,) + shape), np.zeros(shape), L.D2Q9, p)
    h, g = O.run(h, g, L.D2Q9, p, 3000)
    m = O.macroscopic(h, g, L.D2Q9, p)
    np.testing.assert_allclose(m["u"][0].reshape(-1), U * (np.arange(ny) + 0.5) / ny, atol=1e-7 * U)
    assert np.abs(m["phi"] - 1.0).max() < 1e-12
    assert np.abs(m["u"][1]).max() < 1e-12


def test_sliding_walls_exchange_no_phi():
    """Tangentially moving walls hand over momentum, not phi or mass."""
    shape = (1, 12, 10)
    phi, u, P = I.smooth_random(shape, 31, dim=2)
    wu = ((0.0, 0.0, 0.0),) * 2 + ((0.02, 0.0, 0.0), (-0.01, 0.0, 0.0)) + ((0.0, 0.0, 0.0),) * 2
    p = O.Params(M=0.1, W=3.0, sigma=0.01, rho_L=0.01, rho_H=1.0, nu_L=0.1, nu_H=0.05,
                 bc=("periodic", "wall", "periodic"), wall_u=wu)
    h, g = O.init_populations(phi, u, P, L.D2Q9, p)
    phi0 = O.order_parameter(h).sum()
    h, g = O.run(h, g, L.D2Q9, p, 50)
    assert abs(O.order_parameter(h).sum() - phi0) < 1e-12 * phi0


@pytest.mark.slow
def test_layered_couette():
    # the corrected model follows the quadrature whichever wall slides
    assert _couette(1000.0, True, "water")[0] < 0.03
    assert _couette(1000.0, True, "air")[0] < 0.035
    assert _couette(100.0, True, "water")[0] < 0.01
    # without Eq. 13 the water-side sliding wall shows the interface peak the
    # paper reports, while an air-side sliding wall hides it (Section 3)
    err_w, dphi = _couette(100.0, False, "water")
    assert err_w > 0.2 and dphi < 1e-9
    assert _couette(100.0, False, "air")[0] < 0.035


@pytest.mark.parametrize("nx,ny,W,amp", [(150, 600, 2.5, 0.1), (64, 256, 4.0, 0.2), (150, 600, 2.5, 0.0)])
def test_rt_fronts_of_the_initial_interface(nx, ny, W, amp):
    """The Rayleigh-Taylor front diagnostic on the unevolved start: a cosine
    of amplitude amp L puts the spike tip amp L below and the bubble tip
    amp L above the mean interface, to within one row (fronts are whole rows
    where phi crosses 1/2)."""
    s, b = D.rt_fronts(I.perturbed_interface(nx, ny, W, amplitude=amp), nx, ny)
    assert abs(s * nx + amp * nx) <= 1.0 and abs(b * nx - amp * nx) <= 1.0
    assert s <= b + 1.0 / nx


def test_hydrostatic_start_balances_the_body_force():
    """Reading R17: the hydrostatic start's pressure differences along g are
    the trapezoid means of F = (rho - rho_bar) g, its mean is zero, and a
    stable flat layering (heavy below) started from it stays at rest far
    better than one started from P = 0 (a wrong sign or axis would not)."""
    nx, ny, G = 8, 64, 1e-4
    p = O.Params(M=0.05, W=4.0, sigma=1e-3, rho_L=1e-2, rho_H=1.0, nu_L=0.1, nu_H=0.02,
                 g=(0.0, -G, 0.0), force_mode=1, bc=("periodic", "wall", "periodic"))
    phi, _, _ = I.layers((1, ny, nx), axis=1, split=ny / 2 - 0.5, W=4.0)
    P = O.hydrostatic_pressure(phi, p)
    rho = p.rho_L + phi * p.rho_dif
    F = (rho - O.mean_density(phi, p)) * (-G)
    np.testing.assert_allclose(np.diff(P, axis=1), 0.5 * (F[:, 1:] + F[:, :-1]), rtol=0, atol=1e-15)
    assert abs(P.mean()) < 1e-15
    umax = {}
    for name, P0 in (("hydrostatic", P), ("zero", np.zeros_like(P))):
        q = O.Params(**{**p.__dict__, "rho_bar": None})
        h, g = O.init_populations(phi, np.zeros((3,) + phi.shape), P0, L.D2Q9, q)
        h, g = O.run(h, g, L.D2Q9, q, 200)
        umax[name] = np.abs(O.macroscopic(h, g, L.D2Q9, q)["u"]).max()
    assert umax["hydrostatic"] < 0.05 * umax["zero"], umax


@pytest.mark.parametrize("lat,shape", [(L.D2Q9, (1, 20, 26)), (L.D3Q19, (9, 8, 10))], ids=["D2Q9", "D3Q19"])
def test_buoyancy_force_has_no_net_push(lat, shape):
    """Reading R7, force_mode 1: F = (rho - rho_bar) g with rho_bar the mean
    density of the domain, so on a periodic domain the body force sums to
    zero at every step (phi, hence the mean density, is conserved) and the
    total momentum changes only by the sum of mu grad phi, not by any net
    weight: buoyancy without a push on the whole fluid."""
    phi, u, P = I.smooth_random(shape, 13, dim=lat.dim)
    phi = 0.2 + 0.7 * phi          # mean away from 1/2, so rho_bar differs from the mid-density
    g_acc = (0.0, -2e-5, 0.0) if lat.dim == 2 else (0.0, 0.0, -2e-5)
    p = O.Params(M=0.1, W=3.0, sigma=0.01, rho_L=0.01, rho_H=1.0, nu_L=0.1, nu_H=0.05, g=g_acc, force_mode=1)
    h, g = O.init_populations(phi, u, P, lat, p)
    rho_mean = float(O.density(phi, p).mean())
    assert p.rho_bar == pytest.approx(rho_mean, rel=1e-14)
    for _ in range(2):
        m = O.macroscopic(h, g, lat, p)
        scale = np.abs(m["F"]).sum()
        assert scale > 0
        assert np.abs(m["F"].reshape(3, -1).sum(axis=1)).max() < 1e-13 * scale
        h, g = O.run(h, g, lat, p, 10)

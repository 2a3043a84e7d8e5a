"""The two-population phase-field LB time step, FP64, whole-field numpy loops.

Follows Section 2 of the paper (Eqs. 1-12, the central-difference stencils
and the pressure / momentum recovery after Eq. 12) and the high-order
equilibrium correction of Section 3 (Eq. 13).  The step is taken in the
paper's order, one plain pass per quantity, with no fusion:

    phi = sum_i h_i                                        (after Eq. 4)
    grad phi, lap phi by central differences               (stencils after Eq. 12)
    rho(phi), mu_chm (Eq. 8), 1/tau_mix (Eq. 9), F_ex
    u, P from the g moments                                 (after Eq. 12, Eq. 13)
    Gamma_i (Eq. 3), theta (Eq. 4), h_eq (Eq. 2), h BGK collision (Eq. 1)
    K_i (Eq. 7), g_eq (Eq. 6) + delta f_eq (Eq. 13), Pi (Eq. 12),
    filtered g collision (Eqs. 10-11)
    pull streaming (left-hand sides of Eqs. 1 and 10), halfway bounce-back

Fields are numpy arrays of shape (nz, ny, nx) (x fastest, so the flat index
is x + nx*(y + ny*z)); vectors have a leading axis of length 3; populations
have a leading axis of length Q.  A D2Q9 field has nz = 1.

Readings (the paper is silent or garbled at these places):

R1  T = 1/3 and the standard weights (see ``lattice``).
R2  rho(phi) = rho_L + phi*(rho_H - rho_L), rho_dif = rho_H - rho_L: Eq. 9
    puts water (the heavy phase) at phi = 1.
R3  Eq. 12 prints "g_l - G^neq_l"; matching Eq. 10 to the BGK form Eq. 5 as
    the text after Eq. 12 instructs gives G^eq_i = g^eq_i + K_i and
    Pi = sum_l c_l c_l (g_l - g^eq_l).
R4  The "modification of definition of velocity" of Section 3 is not
    written out.  delta f^eq adds u*lap(rho)/4 to the first moment, so the
    velocity is read from (rho + lap(rho)/4) u = sum_i c_i g_i +
    (mu grad phi + F)/2, which keeps sum_i c_i (g_i - g^eq_i) = 0.
    ``modified_velocity=False`` gives rho u = ... instead.
R5  delta f^eq enters g^eq only (it carries lap rho).
R6  Order in a step: phi -> stencils -> rho, mu -> u -> P -> collisions,
    h^eq uses the same u.
R7  F_ex is a force density: F = rho g (force_mode 0) or
    F = (rho - rho_bar) g (force_mode 1, rho_bar the domain mean).
R8  phi is clipped to [0, 1] inside 1/tau_mix only.
R9  Walls: halfway bounce-back for h and g; the phi value at a ghost node
    behind a wall is the adjacent fluid node's (zero normal gradient).
R10 Initialisation: h = h^eq, g = g^eq of the given (phi, u, P).
R17 A buoyancy-driven start at rest takes the hydrostatic pressure,
    grad P = F (``hydrostatic_pressure``); the paper gives no initial
    pressure for its Rayleigh-Taylor cases.
R19 Rebuilding populations from macroscopic fields (the learned warm start
    of this library; the paper has none): g = g^eq + Phi_i : Pi(1) with the
    Chapman-Enskog estimate Pi(1) = -tau_mix T rho (grad u + grad u^T) of the
    non-equilibrium momentum flux, the part the filtered collision (Eq. 10)
    keeps; h = h^eq.
R18 The diffusion correction of Eq. 14 (Section 3) leaves the constant C and
    the function F open, asking only that F vanish on "decent" drops and
    bubbles.  Reading: F(phi, lap phi) = -W^2 max(0, (2 phi - 1) lap phi).
    On the tanh profile phi'' = (16/W^2) phi (1 - phi) (1 - 2 phi), so
    (2 phi - 1) phi'' <= 0 everywhere and F = 0; a dense bubble (a dip of phi
    inside the heavy phase, phi > 1/2, lap phi > 0) or a rarefied droplet (a
    bump inside the light phase, phi < 1/2, lap phi < 0) gives F < 0.  With
    theta + delta theta in h^eq the interface flux becomes
    M (1 - C F) grad phi - theta T n: for C > 0 the correction adds
    diffusion exactly where such structures sit.  C = 0 (the default) is the
    model of Section 2.
"""
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from .lattice import T, Lattice

PERIODIC = "periodic"
WALL = "wall"


@dataclass
class Params:
    """Model parameters in lattice units (Delta x = Delta t = 1)."""
    M: float = 0.1            # mobility (Eq. 1)
    W: float = 4.0            # interface thickness (Eq. 4)
    sigma: float = 0.01       # surface tension (Eq. 8)
    rho_L: float = 0.001      # light phase (air), phi = 0
    rho_H: float = 1.0        # heavy phase (water), phi = 1
    nu_L: float = 0.1 / 6.0   # kinematic viscosity of the light phase
    nu_H: float = 0.1 / 6.0   # kinematic viscosity of the heavy phase
    g: Sequence[float] = (0.0, 0.0, 0.0)   # body acceleration
    force_mode: int = 0       # R7
    rho_bar: Optional[float] = None        # mean density for force_mode 1
    eps: float = 1e-10        # Section 2, after Eq. 4
    modified_velocity: bool = True         # R4
    hocorr: bool = True       # Eq. 13 on/off
    collision: str = "filtered"            # "filtered" (Eq. 10) or "bgk" (Eq. 5)
    bc: Sequence[str] = (PERIODIC, PERIODIC, PERIODIC)   # per axis x, y, z
    # velocity of the wall at each end of each walled axis, wall_u[2 a + side]
    # (side 0: below coordinate 0, side 1: above n_a - 1); R15
    wall_u: Sequence[Sequence[float]] = ((0.0, 0.0, 0.0),) * 6
    C_dtheta: float = 0.0     # constant C of the diffusion correction (Eq. 14, R18)

    @property
    def rho_dif(self):
        return self.rho_H - self.rho_L

    @property
    def tau_phi(self):
        """Relaxation time of the h-LB, Eq. 1: (M/T) + 0.5."""
        return self.M / T + 0.5

    @property
    def tau_L(self):
        """tau_air from nu_air (Section 2, after Eq. 9): nu = T (tau - 1/2)."""
        return self.nu_L / T + 0.5

    @property
    def tau_H(self):
        return self.nu_H / T + 0.5


# --------------------------------------------------------------------------
# neighbour access and streaming
# --------------------------------------------------------------------------
AXES = (2, 1, 0)   # array axis of x, y, z in a (nz, ny, nx) field


def value_at_offset(f, c, bc):
    """f(x + c) on the grid: periodic wrap, or the mirrored fluid node behind
    a wall (R9: zero normal gradient, i.e. the index is clamped)."""
    out = f
    for a in range(3):
        if c[a] == 0:
            continue
        ax = AXES[a] + (f.ndim - 3)
        n = f.shape[ax]
        idx = np.arange(n) + c[a]
        if bc[a] == PERIODIC:
            idx = idx % n
        else:
            idx = np.clip(idx, 0, n - 1)
        out = np.take(out, idx, axis=ax)
    return out


def moving_wall_terms(lat: Lattice, p: Params, s, shape):
    """R15 (reading; the paper assigns wall velocities in its Couette flow of
    Section 3 without writing the boundary rule): a population f*_j that
    leaves x towards a wall moving with u_w returns reduced by the momentum
    the wall hands over, 2 w_j s (c_j . u_w) / T, where s is the density the
    equilibrium carries velocity with (phi for h, rho for g) at x.  Returns
    term[j] on the grid; where x + c_j crosses two walls (a corner) u_w is the
    mean of theirs."""
    nz, ny, nx = shape
    coords = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xyz = (coords[2], coords[1], coords[0])
    n = (nx, ny, nz)
    term = np.zeros((lat.Q,) + tuple(shape))
    for j in range(lat.Q):
        c = lat.c[j]
        usum = np.zeros((3,) + tuple(shape))
        count = np.zeros(shape)
        for a in range(3):
            if c[a] == 0 or p.bc[a] != WALL:
                continue
            t = xyz[a] + c[a]
            for side, hit in ((0, t < 0), (1, t >= n[a])):
                uw = np.asarray(p.wall_u[2 * a + side], dtype=float)
                usum += hit[None] * uw[:, None, None, None]
                count += hit
        cu = np.einsum("a,axyz->xyz", c.astype(float), usum) / np.maximum(count, 1)
        term[j] = 2.0 * lat.w[j] * s * cu / T
    return term


def stream(fstar, lat: Lattice, bc, wall_term=None):
    """Pull streaming, the left-hand sides of Eqs. 1 and 10:
    f_i(x, t+1) = f*_i(x - c_i, t).  If x - c_i lies behind a wall the
    population that left x towards the wall returns reversed (halfway
    bounce-back, R9): f_i(x, t+1) = f*_opp(i)(x, t), less wall_term[opp(i)]
    at x for a moving wall (R15)."""
    nz, ny, nx = fstar.shape[1:]
    coords = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xyz = (coords[2], coords[1], coords[0])
    out = np.empty_like(fstar)
    for i in range(lat.Q):
        c = lat.c[i]
        pulled = fstar[i]
        blocked = np.zeros((nz, ny, nx), dtype=bool)
        for a in range(3):
            if c[a] == 0:
                continue
            ax = AXES[a]
            pulled = np.roll(pulled, c[a], axis=ax)      # pulled[x] = f[x - c]
            if bc[a] == WALL:
                src = xyz[a] - c[a]
                blocked |= (src < 0) | (src >= fstar.shape[1 + ax])
        back = fstar[lat.opp[i]] if wall_term is None else fstar[lat.opp[i]] - wall_term[lat.opp[i]]
        out[i] = np.where(blocked, back, pulled)
    return out


# --------------------------------------------------------------------------
# local quantities
# --------------------------------------------------------------------------
def order_parameter(h):
    """phi = sum_i h_i (Section 2, after Eq. 4)."""
    return h.sum(axis=0)


def gradient(phi, lat: Lattice, bc):
    """Central difference gradient (stencil after Eq. 12):
    grad phi = sum_i {phi(x + c_i) - phi(x - c_i)} c_i w_i / (2T)."""
    gr = np.zeros((3,) + phi.shape)
    for i in range(lat.Q):
        c = lat.c[i]
        diff = value_at_offset(phi, c, bc) - value_at_offset(phi, -c, bc)
        for a in range(3):
            gr[a] += diff * c[a] * lat.w[i]
    return gr / (2.0 * T)


def laplacian(phi, lat: Lattice, bc):
    """Central difference Laplacian (stencil after Eq. 12):
    lap phi = 2 sum_i {phi(x + c_i) - phi(x)} w_i / T."""
    lap = np.zeros(phi.shape)
    for i in range(lat.Q):
        lap += (value_at_offset(phi, lat.c[i], bc) - phi) * lat.w[i]
    return 2.0 * lap / T


def density(phi, p: Params):
    """rho(phi), reading R2."""
    return p.rho_L + phi * p.rho_dif


def chemical_potential(phi, lap, p: Params):
    """Eq. 8: mu = 48 sigma/W phi (phi - 1)(phi - 0.5) - (3 sigma W / 2) lap phi."""
    return (48.0 * p.sigma / p.W) * phi * (phi - 1.0) * (phi - 0.5) \
        - 1.5 * p.sigma * p.W * lap


def inv_tau_mix(phi, p: Params):
    """Eq. 9, harmonic interpolation of the relaxation time, phi clipped (R8)."""
    pc = np.clip(phi, 0.0, 1.0)
    return 1.0 / p.tau_L + pc * (1.0 / p.tau_H - 1.0 / p.tau_L)


def external_force(rho, p: Params):
    """F_ex as a force density (R7)."""
    g = np.asarray(p.g, dtype=np.float64).reshape(3, 1, 1, 1)
    if p.force_mode == 0:
        return g * rho[None]
    return g * (rho - p.rho_bar)[None]


def theta(phi, p: Params):
    """Eq. 4: theta = (M/T) (1 - 4 (phi - 0.5)^2) / W."""
    return (p.M / T) * (1.0 - 4.0 * (phi - 0.5) ** 2) / p.W


def delta_theta(phi, grad, lap, p: Params):
    """Eq. 14: delta theta = C (M/T) F(phi, lap phi) |grad phi|, with F of
    reading R18, F = -W^2 max(0, (2 phi - 1) lap phi)."""
    F = -(p.W ** 2) * np.maximum(0.0, (2.0 * phi - 1.0) * lap)
    mag = np.sqrt((grad ** 2).sum(axis=0))
    return p.C_dtheta * (p.M / T) * F * mag


def normal(grad, p: Params):
    """n = grad phi / (|grad phi| + eps) (Section 2, after Eq. 4)."""
    mag = np.sqrt((grad ** 2).sum(axis=0))
    return grad / (mag + p.eps)


def gamma(u, lat: Lattice):
    """Eq. 3: Gamma_i = w_i {1 + c.u/T + (c.u)^2/(2T^2) - u^2/(2T)}."""
    usq = (u ** 2).sum(axis=0)
    G = np.empty((lat.Q,) + u.shape[1:])
    for i in range(lat.Q):
        cu = sum(lat.c[i][a] * u[a] for a in range(3))
        G[i] = lat.w[i] * (1.0 + cu / T + cu ** 2 / (2.0 * T * T) - usq / (2.0 * T))
    return G


def velocity(g, rho, lap, mu, grad, F, lat: Lattice, p: Params):
    """Momentum recovery after Eq. 12: rho u = sum_i c_i g_i + (mu grad phi + F)/2,
    with the density on the left replaced by rho + lap(rho)/4 when the
    high-order correction is on (reading R4)."""
    J = np.zeros((3,) + rho.shape)
    for i in range(lat.Q):
        for a in range(3):
            if lat.c[i][a] != 0:
                J[a] += lat.c[i][a] * g[i]
    J += 0.5 * (mu[None] * grad + F)
    rho_eff = rho.copy()
    if p.hocorr and p.modified_velocity:
        rho_eff = rho + 0.25 * p.rho_dif * lap
    return J / rho_eff[None]


def pressure(g, u, grad, p: Params):
    """Pressure recovery after Eq. 12: P = T sum_i g_i + (T rho_dif / 2) u . grad phi."""
    return T * g.sum(axis=0) + 0.5 * T * p.rho_dif * (u * grad).sum(axis=0)


def macroscopic(h, g, lat: Lattice, p: Params):
    """All local quantities of a node at time t from the pre-collision
    populations, in the order of reading R6."""
    phi = order_parameter(h)
    grad = gradient(phi, lat, p.bc)
    lap = laplacian(phi, lat, p.bc)
    rho = density(phi, p)
    mu = chemical_potential(phi, lap, p)
    F = external_force(rho, p)
    u = velocity(g, rho, lap, mu, grad, F, lat, p)
    P = pressure(g, u, grad, p)
    return dict(phi=phi, grad=grad, lap=lap, rho=rho, mu=mu, F=F, u=u, P=P)


# --------------------------------------------------------------------------
# equilibria and forcing
# --------------------------------------------------------------------------
def h_equilibrium(phi, u, grad, lat: Lattice, p: Params, G=None, lap=None):
    """Eq. 2: h^eq_i = phi Gamma_i + theta w_i (c_i . n), with theta corrected
    by delta theta of Eq. 14 when C != 0 (R18; lap = lap phi is then needed)."""
    if G is None:
        G = gamma(u, lat)
    n = normal(grad, p)
    th = theta(phi, p)
    if p.C_dtheta != 0.0:
        th = th + delta_theta(phi, grad, lap, p)
    heq = np.empty_like(G)
    for i in range(lat.Q):
        cn = sum(lat.c[i][a] * n[a] for a in range(3))
        heq[i] = phi * G[i] + th * lat.w[i] * cn
    return heq


def forcing(u, grad, mu, F, lat: Lattice, p: Params, G=None):
    """Eq. 7: K_i = {(Gamma_i - w_i) rho_dif + Gamma_i mu / T} (c_i - u) . grad phi
    + Gamma_i (c_i - u) . F / T."""
    if G is None:
        G = gamma(u, lat)
    K = np.empty_like(G)
    for i in range(lat.Q):
        cmu_grad = sum((lat.c[i][a] - u[a]) * grad[a] for a in range(3))
        cmu_F = sum((lat.c[i][a] - u[a]) * F[a] for a in range(3))
        K[i] = ((G[i] - lat.w[i]) * p.rho_dif + G[i] * mu / T) * cmu_grad \
            + G[i] * cmu_F / T
    return K


def high_order_correction(u, lap, lat: Lattice, p: Params):
    """Eq. 13: delta f^eq_i = w_i (c_i . u) lap(rho) / (4T), lap rho = rho_dif lap phi."""
    lap_rho = p.rho_dif * lap
    d = np.empty((lat.Q,) + lap.shape)
    for i in range(lat.Q):
        cu = sum(lat.c[i][a] * u[a] for a in range(3))
        d[i] = lat.w[i] * cu * lap_rho / (4.0 * T)
    return d


def g_equilibrium(rho, u, P, K, lap, lat: Lattice, p: Params, G=None):
    """Eq. 6 plus Eq. 13: g^eq_i = rho Gamma_i + w_i (P/T - rho) - K_i/2 (+ delta f^eq_i)."""
    if G is None:
        G = gamma(u, lat)
    geq = np.empty_like(G)
    for i in range(lat.Q):
        geq[i] = rho * G[i] + lat.w[i] * (P / T - rho) - 0.5 * K[i]
    if p.hocorr:
        geq += high_order_correction(u, lap, lat, p)
    return geq


def second_moment(f, lat: Lattice):
    """sum_l c_l c_l f_l as a (3, 3, ...) tensor (Eq. 12 with f = g - g^eq)."""
    Pi = np.zeros((3, 3) + f.shape[1:])
    for l in range(lat.Q):
        c = lat.c[l]
        for a in range(3):
            for b in range(3):
                if c[a] * c[b] != 0:
                    Pi[a, b] += c[a] * c[b] * f[l]
    return Pi


def hermite_projection(Pi, lat: Lattice):
    """Phi_i : Pi with Phi_i = w_i / (2 T^2) (c_i c_i - T I) (Eq. 11)."""
    trace = Pi[0, 0] + Pi[1, 1] + Pi[2, 2]
    out = np.empty((lat.Q,) + Pi.shape[2:])
    for i in range(lat.Q):
        c = lat.c[i]
        ccPi = sum(c[a] * c[b] * Pi[a, b] for a in range(3) for b in range(3))
        out[i] = lat.w[i] / (2.0 * T * T) * (ccPi - T * trace)
    return out


# --------------------------------------------------------------------------
# collision, step, initialisation
# --------------------------------------------------------------------------
def collide(h, g, lat: Lattice, p: Params, m=None):
    """Post-collision h*, g* at every node (right-hand sides of Eqs. 1 and 10)."""
    if m is None:
        m = macroscopic(h, g, lat, p)
    G = gamma(m["u"], lat)
    # h: Eq. 1 with Eq. 2
    heq = h_equilibrium(m["phi"], m["u"], m["grad"], lat, p, G, m["lap"])
    hstar = h - (h - heq) / p.tau_phi
    # g: Eqs. 6, 7, 13, then Eq. 10 (filtered) or Eq. 5 (BGK)
    K = forcing(m["u"], m["grad"], m["mu"], m["F"], lat, p, G)
    geq = g_equilibrium(m["rho"], m["u"], m["P"], K, m["lap"], lat, p, G)
    omega = inv_tau_mix(m["phi"], p)
    if p.collision == "bgk":
        gstar = g - (g - geq) * omega[None] + K
    else:
        Pi = second_moment(g - geq, lat)                       # Eq. 12, R3
        gstar = geq + K + (1.0 - omega)[None] * hermite_projection(Pi, lat)
    return hstar, gstar


def step(h, g, lat: Lattice, p: Params):
    """One time step: collide at every node, then pull-stream."""
    hstar, gstar = collide(h, g, lat, p)
    if not any(any(v != 0.0 for v in u) for u in p.wall_u):
        return stream(hstar, lat, p.bc), stream(gstar, lat, p.bc)
    phi = hstar.sum(axis=0)            # Eq. 1 conserves phi through the collision
    shape = phi.shape
    return (stream(hstar, lat, p.bc, moving_wall_terms(lat, p, phi, shape)),
            stream(gstar, lat, p.bc, moving_wall_terms(lat, p, density(phi, p), shape)))


def run(h, g, lat: Lattice, p: Params, n):
    for _ in range(n):
        h, g = step(h, g, lat, p)
    return h, g


def mean_density(phi, p: Params):
    """rho_bar of reading R7 from the (conserved) order parameter."""
    return p.rho_L + p.rho_dif * float(phi.mean())


def hydrostatic_pressure(phi, p: Params):
    """Reading R17, a start at rest for buoyancy-driven cases: the pressure
    in balance with the body force, grad P = F (force_mode 1: F = (rho -
    rho_bar) g), integrated along the one axis g points along by the
    trapezoid rule and shifted to zero mean.  phi is (nz, ny, nx).  With P = 0
    instead the unbalanced force launches pressure waves; at density ratio
    1000 they wreck the Rayleigh-Taylor case of Section 4 before t* = 0.25."""
    comps = [a for a in range(3) if p.g[a] != 0.0]
    if len(comps) != 1 or p.force_mode != 1:
        raise ValueError("hydrostatic start: force_mode 1 with g along one axis")
    a = comps[0]
    axis = 2 - a                       # array axes are (z, y, x)
    rho_bar = p.rho_bar if p.rho_bar is not None else mean_density(phi, p)
    F = (density(phi, p) - rho_bar) * p.g[a]
    P = np.cumsum(F, axis=axis) - 0.5 * F - 0.5 * np.take(F, [0], axis=axis)
    return P - P.mean()


def chapman_enskog_pi(phi, u, lat: Lattice, p: Params):
    """Reading R19 (for rebuilding populations from macroscopic fields; the
    paper does not rebuild states): the first-order non-equilibrium second
    moment of g, Pi(1) = -tau_mix T rho (grad u + grad u^T), with grad u by
    the central differences of Section 2 applied to each velocity component
    and tau_mix from Eq. 9.  Returns a (3, 3, ...) tensor."""
    du = np.stack([gradient(u[b], lat, p.bc) for b in range(3)], axis=1)   # du[a, b] = d_a u_b
    tau = 1.0 / inv_tau_mix(phi, p)
    coef = -tau * T * density(phi, p)
    return coef[None, None] * (du + np.swapaxes(du, 0, 1))


def init_populations(phi, u, P, lat: Lattice, p: Params, nonequilibrium=False):
    """Reading R10: h = h^eq(phi, u), g = g^eq(phi, u, P) with the stencils of the
    given phi.  With `nonequilibrium` (R19) g also carries the filtered
    non-equilibrium part Phi_i : Pi(1) of Eq. 11, Pi(1) the Chapman-Enskog
    estimate of chapman_enskog_pi.  Returns (h, g), pre-collision populations
    at t = 0."""
    if p.force_mode == 1 and p.rho_bar is None:
        p.rho_bar = mean_density(phi, p)
    grad = gradient(phi, lat, p.bc)
    lap = laplacian(phi, lat, p.bc)
    rho = density(phi, p)
    mu = chemical_potential(phi, lap, p)
    F = external_force(rho, p)
    G = gamma(u, lat)
    h = h_equilibrium(phi, u, grad, lat, p, G, lap)
    K = forcing(u, grad, mu, F, lat, p, G)
    g = g_equilibrium(rho, u, P, K, lap, lat, p, G)
    if nonequilibrium:
        g = g + hermite_projection(chapman_enskog_pi(phi, u, lat, p), lat)
    return h, g


# --------------------------------------------------------------------------
# 2-D convenience: a D2Q9 field (ny, nx) is the 3-D field (1, ny, nx)
# --------------------------------------------------------------------------
def as3d_scalar(f):
    f = np.asarray(f, dtype=np.float64)
    return f[None] if f.ndim == 2 else f


def as3d_vector(v):
    v = np.asarray(v, dtype=np.float64)
    if v.ndim == 3:              # (2, ny, nx) -> (3, 1, ny, nx)
        out = np.zeros((3, 1) + v.shape[1:])
        out[: v.shape[0], 0] = v
        return out
    return v

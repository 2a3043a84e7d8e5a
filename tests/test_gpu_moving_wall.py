"""Sliding walls (lbm_set_wall_velocity) on the GPU against the FP64 oracle
(oracle R15: halfway bounce-back less the wall's momentum, phi for h and
rho(phi) for g).

* FP64 populations after tens of steps, D2Q9 and D3Q19, both ends of the
  walled axis sliding with different velocities, through the library's FP64
  tile (one-node kernel: 8 for D3Q19, 1 for D2Q9), the bulk-copy tile and
  (D2Q9) a grid of a batch: 1e-10 normwise (operation order only);
* the same in FP32 through the cp.async tile (7): 1e-5 normwise;
* the layered Couette flow of Section 3 in FP32 against the quadrature of
  (eta u')' = 0: within 3 % of the wall speed, as the oracle;
* argument errors."""
import numpy as np
import pytest
from scipy.integrate import cumulative_trapezoid

from oracle import pflbm as O
from paper_1812_00118_gb300 import inputs as I
from parity_helpers import normwise, oracle_lattice, oracle_macro_flat, user_velocity

pytestmark = pytest.mark.gpu
T = 1.0 / 3.0


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00118_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


def oracle_params(prm, bc_user, lat_id, wall_u):
    names = {0: "periodic", 1: "wall"}
    bc = [names[b] for b in bc_user] + ["periodic"] * (3 - len(bc_user))
    return O.Params(M=prm.M, W=prm.W, sigma=prm.sigma, rho_L=prm.rho_L, rho_H=prm.rho_H, nu_L=prm.nu_L,
                    nu_H=prm.nu_H, g=(prm.g[0], prm.g[1], prm.g[2] if lat_id == 1 else 0.0),
                    force_mode=prm.force_mode, eps=prm.eps, bc=tuple(bc), wall_u=wall_u)


# (lattice, oracle shape zyx, user bc, walled user axis, (low wall u, high wall u) in user components)
CASES = [
    (0, (1, 24, 20), (0, 1), 1, ((0.01, 0.0), (-0.02, 0.0))),
    (1, (9, 12, 10), (0, 1, 0), 1, ((0.01, 0.0, -0.005), (0.0, 0.0, 0.02))),
]


def run_case(L, lat_id, shape, bc, axis, walls, steps, tile=None, batch=False, store=None):
    nz, ny, nx = shape
    phi, u, P = I.smooth_random(shape, 41, dim=2 if lat_id == 0 else 3)
    prm = L.make_params(M=0.1, W=3.0, sigma=0.01, rho_L=0.01, rho_H=1.0, nu_L=0.1, nu_H=0.05,
                        store=L.F64 if store is None else store, g_scale=1e3 if store == L.F16S else 0.0)
    user = (nx, ny) if lat_id == 0 else (nx, ny, nz)
    if batch:
        b = L.Batch([user], prm, bcs=[bc])
        sim = b.grid(0)
    else:
        b = None
        sim = L.Simulation(lat_id, user, prm, bc=bc, ghost_band=tile is not None and tile[0] == 4)
        if tile is not None:
            sim.set_tile(*tile)
    for side in (0, 1):
        sim.set_wall_velocity(axis, side, walls[side])
    sim.init_fields(np.ascontiguousarray(phi.reshape(-1)), user_velocity(u, lat_id), np.ascontiguousarray(P.reshape(-1)))
    (b.step if batch else sim.step)(steps)
    out = sim.macro()
    # oracle: wall_u[2 a + side] in oracle (x, y, z) components
    wu = [(0.0, 0.0, 0.0)] * 6
    for side in (0, 1):
        v = list(walls[side]) + [0.0] * (3 - len(walls[side]))
        wu[2 * axis + side] = tuple(v[:3])
    lat = oracle_lattice(lat_id)
    p = oracle_params(prm, bc, lat_id, tuple(wu))
    h, g = O.init_populations(phi, u, P, lat, p)
    h, g = O.run(h, g, lat, p, steps)
    return out, oracle_macro_flat(h, g, lat, p, lat_id), b


PATHS = [(c, path) for c in range(len(CASES)) for path in ("default", "bulkcopy", "batch", "async", "f16s")
         if not (path == "batch" and CASES[c][0] == 1)]   # batches hold D2Q9 grids


@pytest.mark.parametrize("case,path", PATHS, ids=[f"{('d2q9', 'd3q19')[CASES[c][0]]}-{p}" for c, p in PATHS])
def test_sliding_walls_against_oracle(lbm, case, path):
    lat_id, shape, bc, axis, walls = CASES[case]
    tile = {"bulkcopy": (4, 3), "async": (7, 5)}.get(path)
    store = {"async": lbm.F32, "f16s": lbm.F16S}.get(path, lbm.F64)
    (f, Pg, ru), (fo, Po, ruo), _ = run_case(lbm, lat_id, shape, bc, axis, walls, 40, tile=tile,
                                             batch=path == "batch", store=store)
    # FP16-shifted storage (default tile, the wall term written in the units of
    # the stored values): its 11-bit rounding bounds the agreement, while the
    # wall-driven momentum is what rho u mostly is, so a wrong scale or sign of
    # the wall term would be off by its own size
    tol = {"async": 1e-5, "f16s": 2e-2}.get(path, 1e-10)
    errs = (normwise(f, fo), normwise(Pg, Po), normwise(ru, ruo))
    print(path, "errors phi, P, rho u:", errs)
    assert max(errs) < tol, errs


def test_layered_couette_f32(lbm):
    ny, W, U, ratio = 32, 2.5, 1e-3, 1000.0
    prm = lbm.make_params(M=0.1, W=W, sigma=0.01, rho_L=1.0 / ratio, rho_H=1.0, nu_L=0.17 * ratio / 100.0,
                          nu_H=0.17, store=lbm.F32)
    sim = lbm.Simulation(lbm.D2Q9, (1, ny), prm, bc=(lbm.PERIODIC, lbm.WALL))
    sim.set_wall_velocity(1, 0, (U, 0.0))   # the water-side wall slides
    phi, u, P = I.layers((1, ny, 1), axis=1, split=ny / 2 - 0.5, W=W)
    sim.init_fields(phi.reshape(-1).copy(), np.zeros(2 * ny), np.zeros(ny))
    sim.step(6000)
    f, Pg, ru = sim.macro()
    rho = prm.rho_L + f * (prm.rho_H - prm.rho_L)
    ux = ru[:ny] / rho
    y = np.linspace(-0.5, ny - 0.5, 40001)
    phif = 0.5 + 0.5 * np.tanh(2 * ((ny / 2 - 0.5) - y) / W)
    rhof = prm.rho_L + phif * (prm.rho_H - prm.rho_L)
    tL, tH = prm.nu_L / T + 0.5, prm.nu_H / T + 0.5
    om = 1 / tL + phif * (1 / tH - 1 / tL)
    eta = rhof * T * (1 / om - 0.5)
    B = cumulative_trapezoid(1 / eta, y, initial=0.0)
    ua = U * (1.0 - B / B[-1])
    err = np.abs(ux - np.interp(np.arange(ny), y, ua)).max() / U
    assert err < 0.03, err


def test_wall_velocity_argument_errors(lbm):
    prm = lbm.make_params(store=lbm.F32)
    sim = lbm.Simulation(lbm.D2Q9, (8, 8), prm, bc=(lbm.PERIODIC, lbm.WALL))
    for axis, side, u in ((0, 0, (0.0, 0.01)),      # periodic axis
                          (1, 0, (0.0, 0.01)),      # normal component
                          (1, 2, (0.01, 0.0)),      # bad side
                          (2, 0, (0.01, 0.0)),      # no third axis in 2-D
                          (1, 1, (float("nan"), 0.0))):
        with pytest.raises(lbm.LbmError) as e:
            sim.set_wall_velocity(axis, side, u)
        assert e.value.code == lbm.EINVAL
    sim.set_wall_velocity(1, 1, (0.01, 0.0))

"""Batches of D2Q9 grids on the GPU (lbm_batch_*): every grid of a batch
steps exactly as it would alone.

* against the FP64 oracle, grid by grid (1e-10 normwise after 30 steps, the
  single-grid bound of the same arithmetic);
* against the same grids run one at a time through lbm_step, and across the
  batch tiles and chunk lengths (FP64: 1e-14 / 1e-13 normwise, contraction
  differences of separately compiled kernels);
* CUDA-graph replays against single launches: bit-exact (same kernel, and
  each node's arithmetic does not depend on which CTA takes its item).
"""
import numpy as np
import pytest

from oracle import pflbm as O
from paper_1812_00118_gb300 import inputs as I
from parity_helpers import normwise, oracle_lattice, oracle_macro_flat, oracle_params, user_velocity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00118_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


# (nx, ny, bc, parameter overrides, drop?)
GRIDS = [
    ((5, 7), (0, 0), dict(), False),
    ((33, 17), (1, 0), dict(rho_L=0.01, nu_L=0.05), True),
    ((130, 9), (0, 1), dict(W=3.0, sigma=0.02), False),
    ((64, 40), (0, 0), dict(rho_L=0.1, nu_L=0.2, nu_H=0.01), True),
    ((2, 3), (0, 0), dict(M=0.05), False),
    ((40, 66), (1, 1), dict(g=(1e-5, -2e-5)), True),
]


def fields(shape, seed, drop):
    nx, ny = shape
    zyx = (1, ny, nx)
    if drop:
        return I.sphere(zyx, (nx / 2 + 0.31, ny / 2 - 0.23, 0), min(nx, ny) / 4, 4.0, drop=True)
    return I.smooth_random(zyx, seed, dim=2)


def make_batch(L, store, grids=GRIDS, g_scale=0.0):
    base = dict(M=0.1, W=4.0, sigma=0.01, rho_L=0.001, rho_H=1.0, nu_L=0.1, nu_H=0.02, store=store, g_scale=g_scale)
    params, init = [], []
    for k, (shape, bc, over, drop) in enumerate(grids):
        kw = dict(base)
        kw.update(over)
        params.append(L.make_params(**kw))
        init.append(fields(shape, 10 + k, drop))
    b = L.Batch([g[0] for g in grids], params, bcs=[g[1] for g in grids])
    for k, (phi, u, P) in enumerate(init):
        b.grid(k).init_fields(np.ascontiguousarray(phi.reshape(-1)), user_velocity(u, 0),
                              np.ascontiguousarray(P.reshape(-1)))
    return b, params, init


def populations(b):
    return [b.grid(k).get_populations() for k in range(len(b))]


def test_batch_against_oracle_f64(lbm):
    b, params, init = make_batch(lbm, lbm.F64)
    b.step(30)
    lat = oracle_lattice(0)
    for k, (shape, bc, _, _) in enumerate(GRIDS):
        phi, u, P = init[k]
        p = oracle_params(params[k], bc, 0)
        h, g = O.init_populations(phi, u, P, lat, p)
        h, g = O.run(h, g, lat, p, 30)
        f, Pg, ru = b.grid(k).macro()
        fo, Po, ruo = oracle_macro_flat(h, g, lat, p, 0)
        assert normwise(f, fo) < 1e-10, k
        assert normwise(Pg, Po) < 1e-10, k
        assert normwise(ru, ruo) < 1e-10, k


def test_batch_equals_grids_alone_f64(lbm):
    b, params, init = make_batch(lbm, lbm.F64)
    b.step(9)
    got = populations(b)
    for k, (shape, bc, _, _) in enumerate(GRIDS):
        sim = lbm.Simulation(lbm.D2Q9, shape, params[k], bc=bc)
        phi, u, P = init[k]
        sim.init_fields(np.ascontiguousarray(phi.reshape(-1)), user_velocity(u, 0), np.ascontiguousarray(P.reshape(-1)))
        sim.step(9)
        h, g = sim.get_populations()
        assert normwise(got[k][0], h) < 1e-14 and normwise(got[k][1], g) < 1e-13, k


@pytest.mark.parametrize("store,g_scale,tol", [("F16S", 1e3, 2e-2), ("BF16S", 0.0, 1e-1)], ids=["f16s", "bf16s"])
def test_batch_16bit_storage(lbm, store, g_scale, tol):
    """16-bit shifted storage in the batch kernel (the collision computes the
    stored shifted and scaled values directly): every grid against the same
    grid stepped alone with the same storage, and against the FP64 oracle,
    after 5 steps.  Both runs round to 16 bits, so they agree to the storage
    rounding rather than bit for bit; a wrong shift or scale would be off by
    the size of the populations themselves."""
    st = getattr(lbm, store)
    b, params, init = make_batch(lbm, st, g_scale=g_scale)
    b.step(5)
    lat = oracle_lattice(0)
    for k, (shape, bc, _, _) in enumerate(GRIDS):
        fb, Pb, rb = b.grid(k).macro()
        sim = lbm.Simulation(lbm.D2Q9, shape, params[k], bc=bc)
        phi, u, P = init[k]
        sim.init_fields(np.ascontiguousarray(phi.reshape(-1)), user_velocity(u, 0), np.ascontiguousarray(P.reshape(-1)))
        sim.step(5)
        fs, Ps, rs = sim.macro()
        sim.close()
        p = oracle_params(params[k], bc, 0)
        h, g = O.init_populations(phi, u, P, lat, p)
        h, g = O.run(h, g, lat, p, 5)
        fo, Po, ruo = oracle_macro_flat(h, g, lat, p, 0)
        for name, a, a1, o in (("phi", fb, fs, fo), ("P", Pb, Ps, Po), ("rho_u", rb, rs, ruo)):
            assert np.isfinite(a).all(), (k, name)
            assert normwise(a, a1) < tol and normwise(a, o) < tol, (k, name, normwise(a, a1), normwise(a, o))


def test_batch_tiles_and_chunks_agree_f64(lbm):
    ref = None
    for tile, lz in ((1, 16), (0, 1), (0, 5), (2, 3), (3, 16), (2, 100), (1, 2)):
        b, _, _ = make_batch(lbm, lbm.F64)
        b.set_tile(tile, lz)
        assert b.get_tile()[:2] == (tile, lz)
        b.step(7)
        pops = populations(b)
        if ref is None:
            ref = pops
            continue
        for k in range(len(GRIDS)):
            assert normwise(pops[k][0], ref[k][0]) < 1e-14 and normwise(pops[k][1], ref[k][1]) < 1e-13, (tile, lz, k)


@pytest.mark.parametrize("store", ["F64", "F32"])
def test_graph_replay_bit_exact(lbm, store):
    st = getattr(lbm, store)
    a, _, _ = make_batch(lbm, st)
    a.step(7)
    b, _, _ = make_batch(lbm, st)
    b.set_graph(3)            # two graph replays (from buffer 0, then buffer 1) and one launch
    n0 = b.launch_count()
    b.step(7)
    assert b.launch_count() - n0 == 7
    b.step(6)                 # replays of both graphs again
    a.step(6)
    for (ha, ga), (hb, gb) in zip(populations(a), populations(b)):
        assert np.array_equal(ha, hb) and np.array_equal(ga, gb)


def test_sequential_launches_match_f64(lbm):
    a, _, _ = make_batch(lbm, lbm.F64)
    a.step(5)
    b, _, _ = make_batch(lbm, lbm.F64)
    n0 = b.launch_count()
    b.step_sequential(5)
    assert b.launch_count() - n0 == 5 * len(GRIDS)
    for (ha, ga), (hb, gb) in zip(populations(a), populations(b)):
        assert normwise(hb, ha) < 1e-14 and normwise(gb, ga) < 1e-13


def test_one_step_f32_against_oracle(lbm):
    """Smooth random grids only: a drop starts from P = 0, u = 0, where one
    step leaves P ~ 1e-24 and a relative comparison measures nothing."""
    b, params, init = make_batch(lbm, lbm.F32)
    b.step(1)
    lat = oracle_lattice(0)
    for k, (shape, bc, _, drop) in enumerate(GRIDS):
        if drop:
            continue
        phi, u, P = init[k]
        p = oracle_params(params[k], bc, 0)
        h, g = O.init_populations(phi, u, P, lat, p)
        h, g = O.step(h, g, lat, p)
        f, Pg, ru = b.grid(k).macro()
        fo, Po, ruo = oracle_macro_flat(h, g, lat, p, 0)
        assert normwise(f, fo) < 1e-5 and normwise(Pg, Po) < 1e-5 and normwise(ru, ruo) < 1e-5, k


def test_autotune_restores_state(lbm):
    b, _, _ = make_batch(lbm, lbm.F32)
    b.step(3)
    before = populations(b)
    tile, lz, ms = b.autotune(2)
    assert 0 <= tile < 4 and lz in (4, 8, 16, 32) and ms > 0
    assert b.get_tile()[:2] == (tile, lz)
    after = populations(b)
    for (h0, g0), (h1, g1) in zip(before, after):
        assert np.array_equal(h0, h1) and np.array_equal(g0, g1)


def test_grid_views_do_not_step(lbm):
    b, _, _ = make_batch(lbm, lbm.F64)
    v = b.grid(1)
    for call in (lambda: v.step(1), lambda: v.set_tile(1, 8), lambda: v.autotune(1), lambda: v.step_profiled(1)):
        with pytest.raises(lbm.LbmError) as e:
            call()
        assert e.value.code == lbm.EINVAL
    assert v.get_tile()[0] == 1
    d = v.diagnostics()
    assert d["nonfinite"] == 0


def test_batch_rejects_bad_input(lbm):
    p32 = lbm.make_params(store=lbm.F32)
    p64 = lbm.make_params(store=lbm.F64)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Batch([(8, 8), (8, 8)], [p32, p64])   # mixed storage
    assert e.value.code == lbm.EINVAL
    b = lbm.Batch([(8, 8)], p32)
    with pytest.raises(lbm.LbmError):
        b.set_tile(4, 8)
    with pytest.raises(lbm.LbmError):
        b.set_tile(0, 0)
    with pytest.raises(lbm.LbmError):
        b.set_graph(-1)
    with pytest.raises(IndexError):
        b.grid(1)

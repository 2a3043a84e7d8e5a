"""Host logic of the batch (no GPU): the work list of lbm_batch_plan covers
every node of every grid exactly once, in the documented order, and rejects
bad arguments."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lbm():
    from paper_1812_00118_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


SHAPES = [(5, 7), (33, 17), (130, 9), (64, 64), (1, 1), (257, 3)]


@pytest.mark.parametrize("tx,lz", [(32, 1), (64, 4), (128, 16), (256, 32), (7, 5)])
def test_plan_covers_each_node_once(lbm, tx, lz):
    items = lbm.plan(SHAPES, tx, lz)
    expect = sum(-(-nx // tx) * -(-ny // lz) for nx, ny in SHAPES)
    assert items.shape == (expect, 4)
    for c, (nx, ny) in enumerate(SHAPES):
        cover = np.zeros((ny, nx), dtype=np.int64)   # internal z = user y
        for _, x0, z0, z1 in items[items[:, 0] == c]:
            assert 0 <= x0 < nx and x0 % tx == 0
            assert 0 <= z0 < z1 <= ny and z0 % lz == 0 and z1 - z0 <= lz
            cover[z0:z1, x0:min(x0 + tx, nx)] += 1
        assert (cover == 1).all()


def test_plan_order(lbm):
    items = lbm.plan(SHAPES, 64, 4)
    # grids in order; within a grid z chunks in order, tile columns in order within a chunk
    key = items[:, 0] * 10**8 + items[:, 2] * 10**4 + items[:, 1]
    assert (np.diff(key) > 0).all()


def test_plan_rejects_bad_arguments(lbm):
    import ctypes
    lib = lbm.load()
    g = lbm._grids([(8, 8)], None)
    assert lib.lbm_batch_plan(1, g, 0, 4, None, 0) == lbm.EINVAL
    assert lib.lbm_batch_plan(1, g, 32, 0, None, 0) == lbm.EINVAL
    assert lib.lbm_batch_plan(0, g, 32, 4, None, 0) == lbm.EINVAL
    g[0].nz = 2   # not a D2Q9 grid
    assert lib.lbm_batch_plan(1, g, 32, 4, None, 0) == lbm.EINVAL
    g[0].nz, g[0].nx = 1, 0
    assert lib.lbm_batch_plan(1, g, 32, 4, None, 0) == lbm.EINVAL
    out = (ctypes.c_int * 4)()
    g[0].nx = 8
    assert lib.lbm_batch_plan(1, g, 32, 4, out, 1) == 2   # total count, first item written
    assert list(out) == [0, 0, 0, 4]

"""Failure detection through the C-ABI, with every failure made on the host:
no GPU fault, trap or hang is provoked.

* A NaN in the phi given to lbm_init_fields: lbm_diagnostics reports
  LBM_EDIVERGED (non-finite fields), lbm_step then refuses to advance the
  state (LBM_EDIVERGED, nothing launched), and a new lbm_init_fields clears
  the condition.
* The bounded waits of the bulk-copy pipeline (tile 4), given a poll limit
  of 0 by the host: every wait gives up at once, the kernel raises the error
  flag, lets its copies in flight land and returns; lbm_diagnostics reports
  LBM_ETIMEOUT, the context stays usable, and a new initialisation with the
  default limit steps normally again.
"""
import numpy as np
import pytest

from paper_1812_00118_gb300 import inputs as I
from parity_helpers import user_velocity

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


def fields(shape=(12, 14, 16)):
    phi, u, P = I.smooth_random(shape, 9)
    return np.ascontiguousarray(phi.reshape(-1)), user_velocity(u, 1), np.ascontiguousarray(P.reshape(-1))


def test_nan_input_diverged_then_recovers(lbm):
    phi, u, P = fields()
    sim = lbm.Simulation(lbm.D3Q19, (16, 14, 12), lbm.make_params(store=lbm.F32))
    bad = phi.copy()
    bad[123] = np.nan
    sim.init_fields(bad, u, P)
    with pytest.raises(lbm.LbmError) as e:
        sim.diagnostics()
    assert e.value.code == lbm.EDIVERGED
    n0 = sim.launch_count()
    with pytest.raises(lbm.LbmError) as e:
        sim.step(3)
    assert e.value.code == lbm.EDIVERGED
    assert sim.launch_count() == n0          # nothing was launched
    sim.init_fields(phi, u, P)
    sim.step(3)
    d = sim.diagnostics()
    assert d["nonfinite"] == 0


def test_pipeline_wait_timeout_reported(lbm):
    phi, u, P = fields((12, 16, 40))
    sim = lbm.Simulation(lbm.D3Q19, (40, 16, 12), lbm.make_params(store=lbm.F32), ghost_band=True)
    try:
        sim.set_tile(4, 4)
    except lbm.LbmError as e:
        assert e.code == lbm.ENOTSUP
        pytest.skip("the bulk-copy tile does not apply to this grid")
    sim.init_fields(phi, u, P)
    sim.set_wait_limit(0)
    sim.step(1)
    with pytest.raises(lbm.LbmError) as e:
        sim.diagnostics()
    assert e.value.code == lbm.ETIMEOUT
    # the context is usable: a new state with the default limit steps normally
    sim.set_wait_limit(1 << 22)
    sim.init_fields(phi, u, P)
    sim.step(5)
    d = sim.diagnostics()
    assert d["nonfinite"] == 0
    with pytest.raises(lbm.LbmError):
        sim.set_wait_limit(-1)

"""Galilean test of Section 3 on the GPU: a 1-D periodic domain of 100 nodes
(a D2Q9 grid one node high), a drop in the centre, u = 0.025 everywhere, one
full revolution (4000 steps).

* FP64 against the oracle after the revolution (1e-9 normwise: operation
  order alone, accumulated over 4000 steps);
* FP32: the advected drop keeps its velocity within 10 % and comes back to
  its initial profile (the modified-velocity reading of Section 3), while
  the uncorrected model (hocorr = 0) does not keep it -- the contrast the
  paper draws."""
import numpy as np
import pytest

from oracle import lattice as OL
from oracle import pflbm as O

pytestmark = pytest.mark.gpu

NX, W, U0, STEPS = 100, 3.0, 0.025, 4000


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00118_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


def fields():
    x = np.arange(NX)
    phi = 0.5 + 0.5 * np.tanh(2 * (20 - np.abs(x - 49.5)) / W)   # centre between nodes
    u = np.zeros((2, NX))
    u[0] = U0
    return phi, u


def params(lbm, store, hocorr=1):
    return lbm.make_params(M=0.1, W=W, sigma=0.01, rho_L=1e-3, rho_H=1.0, nu_L=0.17, nu_H=0.017,
                           hocorr=hocorr, store=store)


def run_gpu(lbm, store, hocorr=1):
    phi, u = fields()
    sim = lbm.Simulation(lbm.D2Q9, (NX, 1), params(lbm, store, hocorr))
    sim.init_fields(phi.copy(), u.reshape(-1).copy(), np.zeros(NX))
    sim.step(STEPS)
    f, P, ru = sim.macro()
    d = sim.diagnostics(raise_on_divergence=False)
    sim.close()
    return f, P, ru, d


def test_galilean_revolution_f64_against_oracle(lbm):
    f, P, ru, _ = run_gpu(lbm, lbm.F64)
    phi, u = fields()
    p = O.Params(M=0.1, W=W, sigma=0.01, rho_L=1e-3, rho_H=1.0, nu_L=0.17, nu_H=0.017)
    shape = (1, 1, NX)
    u3 = np.zeros((3,) + shape)
    u3[0] = U0
    h, g = O.init_populations(phi.reshape(shape), u3, np.zeros(shape), OL.D2Q9, p)
    h, g = O.run(h, g, OL.D2Q9, p, STEPS)
    m = O.macroscopic(h, g, OL.D2Q9, p)
    ref_ru = (m["rho"][None] * m["u"])[:2].reshape(-1)
    for a, b in ((f, m["phi"].reshape(-1)), (P, m["P"].reshape(-1)), (ru, ref_ru)):
        assert np.abs(a - b).max() / np.abs(b).max() < 1e-9


def test_galilean_invariance_f32(lbm):
    f, P, ru, d = run_gpu(lbm, lbm.F32)
    phi0, _ = fields()
    rho = 1e-3 + f * (1.0 - 1e-3)
    ux = ru[:NX] / rho
    assert d["nonfinite"] == 0
    assert np.abs(ux - U0).max() / U0 < 0.10
    # after one revolution the drop is back where it started: circular centroid
    # within 5 % of the period (a pointwise check would see a one-node lag of a
    # W = 3 interface as an O(1) difference)
    ang = 2 * np.pi * np.arange(NX) / NX
    centre = lambda a: np.angle(np.sum(a * np.exp(1j * ang))) * NX / (2 * np.pi)
    shift = (centre(f) - centre(phi0) + NX / 2) % NX - NX / 2
    assert abs(shift) < 0.05 * NX
    assert abs(f.sum() - phi0.sum()) < 1e-5 * phi0.sum()


def test_uncorrected_model_loses_the_velocity(lbm):
    f, P, ru, d = run_gpu(lbm, lbm.F64, hocorr=0)
    rho = 1e-3 + f * (1.0 - 1e-3)
    with np.errstate(all="ignore"):
        dev = np.abs(ru[:NX] / rho - U0).max() / U0
    assert d["nonfinite"] > 0 or not dev < 0.5

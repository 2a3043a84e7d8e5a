"""The allocation-free diagnostics entry point against lbm_diagnostics.

lbm_field_sums_noalloc serves callers that cannot allocate device memory
(a host framework owning all device memory, a loop that must not enter the
allocator): its scratch is a static device array inside the library.
This file is collected last so that, if it fails, every other test has
already run; it passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_field_sums_noalloc_matches_diagnostics():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00118_gb300 import build, inputs as I, lbm
    build.build()
    lbm.load()
    nx, ny, nz = 40, 36, 30
    phi, u, P = I.sphere((nz, ny, nx), (19.5, 17.5, 14.5), 8.0, 4.0, drop=True)
    prm = lbm.make_params(M=0.1, W=4.0, sigma=0.01, rho_L=0.001, rho_H=1.0, nu_L=0.1, nu_H=0.1, store=lbm.F32)
    sim = lbm.Simulation(lbm.D3Q19, (nx, ny, nz), prm)
    sim.init_fields(np.ascontiguousarray(phi.reshape(-1)), np.ascontiguousarray(u.reshape(-1)),
                    np.ascontiguousarray(P.reshape(-1)))
    N = nx * ny * nz
    rho_L, rho_dif = 0.001, 1.0 - 0.001
    for steps in (50, 30):          # two calls in a row, on evolving fields
        sim.step(steps)
        ref = sim.diagnostics()
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        Pd = torch.empty_like(f)
        ru = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        sim.macro(f, Pd, ru)
        rho = rho_L + f * rho_dif
        comps = [ru[k * N:(k + 1) * N] / rho for k in range(3)]
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        lbm.field_sums_noalloc(f, Pd, comps, rho_L, rho_dif, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert o[0] == pytest.approx(ref["sum_phi"], rel=1e-12)
        assert o[1] == pytest.approx(ref["sum_rho"], rel=1e-12)
        assert o[2] == pytest.approx(ref["max_u"], rel=1e-12)
        assert o[3] == ref["nonfinite"] == 0


def test_field_sums_noalloc_rejects_oversize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00118_gb300 import lbm
    lbm.load()
    import ctypes
    f = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lbm.load().lbm_field_sums_noalloc(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()), None,
                                           None, None, lbm.NOALLOC_MAX_NODES + 1, 0.0, 1.0,
                                           ctypes.c_void_p(out.data_ptr()), None)
    assert rc == lbm.EINVAL

"""The checked debugging build (LBM_CHECKED): the step kernels check every
plane's pull offsets and every write offset against the population arrays
and record an offset outside them (lbm_checked_status) instead of using it.

On periodic and walled D3Q19 grids (the default tile, the cp.async and the
bulk-copy tiles) and on a D2Q9 batch, a checked run records nothing and
gives the populations of the default build: FP64 to 1e-12 (the checks touch
only integer offsets; instruction scheduling may still contract a product
differently).  The checked library is built on first use into
_lib/liblbm_checked.so and run in a child process (LBM_CHECKED=1 selects it
in the binding)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_1812_00118_gb300 import lbm as L, inputs as I
lib = L.load()
out = {"checked_build": int(lib.lbm_is_checked_build()), "runs": {}}
def case(lat, shape, bc, tile, steps, store):
    if lat == L.D3Q19:
        nx, ny, nz = shape
        phi, u, P = I.smooth_random((nz, ny, nx), 5)
        ushape = u.reshape(-1)
    else:
        nx, ny = shape
        phi, u, P = I.smooth_random((1, ny, nx), 5, dim=2)
        ushape = np.ascontiguousarray(np.stack([u[0], u[1]]).reshape(-1))
    prm = L.make_params(M=0.1, W=3.0, sigma=0.01, rho_L=0.1, rho_H=1.0, nu_L=0.05, nu_H=0.02, store=store)
    sim = L.Simulation(lat, shape, prm, bc=bc, ghost_band=tile == 4)
    sim.init_fields(np.ascontiguousarray(phi.reshape(-1)), ushape, np.ascontiguousarray(P.reshape(-1)))
    if tile is not None:
        try:
            sim.set_tile(tile, 5)
        except L.LbmError:
            sim.close(); return None
    sim.step(steps)
    h, g = sim.get_populations()
    sim.close()
    return [float(np.abs(h).sum()), float(np.abs(g).sum()), h[::97].tolist(), g[::97].tolist()]
for name, args in [("d3q19_periodic_t8", (L.D3Q19, (13, 21, 37), (L.PERIODIC,) * 3, 8, 7, L.F64)),
                   ("d3q19_walls_t8", (L.D3Q19, (19, 11, 35), (L.WALL, L.PERIODIC, L.WALL), 8, 7, L.F64)),
                   ("d3q19_walls_t7", (L.D3Q19, (19, 11, 35), (L.WALL, L.PERIODIC, L.WALL), 7, 7, L.F32)),
                   ("d3q19_periodic_t4", (L.D3Q19, (32, 16, 24), (L.PERIODIC,) * 3, 4, 7, L.F64)),
                   ("d2q9_walls_t1", (L.D2Q9, (40, 70), (L.WALL, L.WALL), 1, 7, L.F64))]:
    out["runs"][name] = case(*args)
# a batch of D2Q9 grids
b = L.Batch([(24, 20), (17, 33), (40, 8)], L.make_params(M=0.1, W=3.0, sigma=0.01, rho_L=0.1, rho_H=1.0,
                                                        nu_L=0.05, nu_H=0.02, store=L.F64))
for k, (nx, ny) in enumerate([(24, 20), (17, 33), (40, 8)]):
    phi, u, P = I.smooth_random((1, ny, nx), 7 + k, dim=2)
    b.grid(k).init_fields(np.ascontiguousarray(phi.reshape(-1)),
                          np.ascontiguousarray(np.stack([u[0], u[1]]).reshape(-1)), np.ascontiguousarray(P.reshape(-1)))
b.step(6)
vals = []
for k in range(3):
    f, P, ru = b.grid(k).macro()
    vals += [float(f.sum()), float(P.sum())]
b.close()
out["runs"]["batch"] = vals
out["status"] = int(lib.lbm_checked_status(None))
print("RESULT" + json.dumps(out))
"""


def run_child(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT")][-1]
    return json.loads(line[len("RESULT"):])


def test_checked_build_records_nothing_and_matches():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00118_gb300 import build
    build.build()
    build.build(checked=True)
    plain = run_child({"LBM_CHECKED": "0"})
    checked = run_child({"LBM_CHECKED": "1"})
    assert plain["checked_build"] == 0 and checked["checked_build"] == 1
    assert plain["status"] == 0 and checked["status"] == 0
    for name, a in plain["runs"].items():
        b = checked["runs"][name]
        if a is None:
            assert b is None, name
            continue
        a, b = np.concatenate([np.ravel(v) for v in a]), np.concatenate([np.ravel(v) for v in b])
        tol = 1e-6 if "t7" in name else 1e-12
        assert np.allclose(a, b, rtol=tol, atol=tol * np.abs(a).max()), name

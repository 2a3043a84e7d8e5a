"""Writes rt_ratio1000_fronts.txt, the spike and bubble fronts of the density
ratio 1000 Rayleigh-Taylor case of Section 4 at t* = 0.5 and 1, from the FP64
oracle.  Test infrastructure: it runs only oracle/ on the input recipe of
paper_1812_00118_gb300.inputs (about 30 minutes on one core).

    python tests/golden/make_rt1000_fronts.py

Parameters: the paper's 256 x 1000 case (sigma 4.7e-1 for its light density
1 and water density 1000, so 4.7e-4 with the heavy density 1; W 5, M 1.3e-2,
nu_water 4.1e-3, dynamic viscosity ratio 100, g 1e-5 acting on rho - rho_bar,
walls at the top and bottom, periodic sideways).  The fluid starts at rest
in hydrostatic balance (oracle reading R17) with the interface perturbed by
a cosine of amplitude 0.1 L; the paper gives neither.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import diagnostics as D  # noqa: E402
from oracle import lattice as OL  # noqa: E402
from oracle import pflbm as O  # noqa: E402
from paper_1812_00118_gb300 import inputs as I  # noqa: E402

NX, NY, G = 256, 1000, 1e-5
RATIO, SIGMA_PAPER, W, M, NU_W, MU_RATIO = 1000.0, 4.7e-1, 5.0, 1.3e-2, 4.1e-3, 100.0
TSTARS = (0.5, 1.0)


def params():
    return O.Params(M=M, W=W, sigma=SIGMA_PAPER / RATIO, rho_L=1.0 / RATIO, rho_H=1.0,
                    nu_L=NU_W * RATIO / MU_RATIO, nu_H=NU_W, g=(0.0, -G, 0.0), force_mode=1,
                    bc=("periodic", "wall", "periodic"))


def main():
    p = params()
    shape = (1, NY, NX)
    phi0 = I.perturbed_interface(NX, NY, W).reshape(shape)
    P0 = O.hydrostatic_pressure(phi0, p)
    h, g = O.init_populations(phi0, np.zeros((3,) + shape), P0, OL.D2Q9, p)
    t_unit = 1.0 / np.sqrt(G / NX)
    lines = ["# Rayleigh-Taylor, density ratio 1000 (Section 4), 256 x 1000, hydrostatic start: fronts from the FP64 oracle",
             "# written by tests/golden/make_rt1000_fronts.py; columns: t*, steps, spike / L, bubble / L"]
    done = 0
    for ts in TSTARS:
        n = int(round(ts * t_unit))
        for _ in range(n - done):
            h, g = O.step(h, g, OL.D2Q9, p)
        done = n
        phi = O.macroscopic(h, g, OL.D2Q9, p)["phi"]
        if not np.isfinite(phi).all():
            raise SystemExit(f"oracle run not finite at t* = {ts}")
        s, b = D.rt_fronts(phi, NX, NY)
        lines.append(f"{ts} {n} {s:.6f} {b:.6f}")
        print(lines[-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "rt_ratio1000_fronts.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

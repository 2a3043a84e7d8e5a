"""Writes rt_ratio3_fronts.txt, the spike and bubble fronts of the density
ratio 3 Rayleigh-Taylor case of Section 4 at t* = 1 and 2, from the FP64
oracle.  Test infrastructure: it runs only oracle/ on the seeded input
recipe of paper_1812_00118_gb300.inputs (about 12 minutes on one core).

    python tests/golden/make_rt_fronts.py

Parameters: the paper's 150 x 600 case (sigma 8.6e-4, W 2.5, M 5.8e-3,
nu_water 1.9e-3, viscosity ratio 1, g 1e-5 acting on rho - rho_bar, walls at
the top and bottom, periodic sideways).  The paper's densities are light 1,
water 3: its printed capillary number 0.26 = rho_water U nu_water / sigma,
U = sqrt(g L), holds only with those.  The model is unchanged when rho, P and
sigma are scaled together, so with the heavy density 1 used here sigma is
8.6e-4 / 3.
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

NX, NY, G = 150, 600, 1e-5
RATIO, SIGMA_PAPER, W, M, NU_W, MU_RATIO = 3.0, 8.6e-4, 2.5, 5.8e-3, 1.9e-3, 1.0
TSTARS = (1.0, 2.0)


def params():
    return O.Params(M=M, W=W, sigma=SIGMA_PAPER / RATIO, rho_L=1.0 / RATIO, rho_H=1.0,
                    nu_L=NU_W * RATIO / MU_RATIO, nu_H=NU_W, g=(0.0, -G, 0.0), force_mode=1,
                    bc=("periodic", "wall", "periodic"))


def main():
    p = params()
    phi0 = I.perturbed_interface(NX, NY, W)
    shape = (1, NY, NX)
    h, g = O.init_populations(phi0.reshape(shape), np.zeros((3,) + shape), np.zeros(shape), OL.D2Q9, p)
    t_unit = 1.0 / np.sqrt(G / NX)
    lines = ["# Rayleigh-Taylor, density ratio 3 (Section 4), 150 x 600: fronts from the FP64 oracle",
             "# written by tests/golden/make_rt_fronts.py; columns: t*, steps, spike / L, bubble / L"]
    done = 0
    for ts in TSTARS:
        n = int(round(ts * t_unit))
        for _ in range(n - done):
            h, g = O.step(h, g, OL.D2Q9, p)
        done = n
        phi = O.macroscopic(h, g, OL.D2Q9, p)["phi"]
        s, b = D.rt_fronts(phi, NX, NY)
        lines.append(f"{ts} {n} {s:.6f} {b:.6f}")
        print(lines[-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "rt_ratio3_fronts.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

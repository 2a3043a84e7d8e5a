"""Velocity sets of the oracle (Section 2: "the D3Q19 or D2Q9 lattice model").

The paper names the lattices but prints neither the velocities nor the
weights, and uses the lattice temperature T without defining it.  The
oracle takes the standard sets: T = c_s^2 = 1/3, D2Q9 weights 4/9, 1/9,
1/36 and D3Q19 weights 1/3, 1/18, 1/36.  Every velocity is stored with
three components; D2Q9 has c_z = 0, so a 2-D field is a 3-D field with
nz = 1 and the same code path serves both lattices.

This table is the oracle's own; the GPU library defines its own table in
its own order, and tests match the two by velocity vector.
"""
import numpy as np

T = 1.0 / 3.0


class Lattice:
    """A velocity set: c (Q, 3) int, w (Q,) float64, opp (Q,) int."""

    def __init__(self, name, c, w):
        self.name = name
        self.c = np.asarray(c, dtype=np.int64)
        self.w = np.asarray(w, dtype=np.float64)
        self.Q = len(self.w)
        self.dim = 2 if name == "D2Q9" else 3
        # index of the opposite velocity: c_opp[i] = -c_i
        self.opp = np.array([
            next(j for j in range(self.Q) if np.all(self.c[j] == -self.c[i]))
            for i in range(self.Q)
        ])


D2Q9 = Lattice(
    "D2Q9",
    [(0, 0, 0),
     (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0),
     (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)],
    [4.0 / 9.0] + [1.0 / 9.0] * 4 + [1.0 / 36.0] * 4,
)

D3Q19 = Lattice(
    "D3Q19",
    [(0, 0, 0),
     (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
     (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
     (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
     (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)],
    [1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12,
)


def get(name):
    return {"D2Q9": D2Q9, "D3Q19": D3Q19}[name]

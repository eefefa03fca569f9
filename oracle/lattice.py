"""D3Q19 lattice (Sec. II.A, "lattice weights" equation; velocity set of the
standard D3Q19 model the paper uses).  TEST INFRASTRUCTURE ONLY.

Index order (x, y, z components):
  0      rest
  1..6   axis links  +x -x +y -y +z -z          (the D3Q7 subset "Q6")
  7..18  face diagonals
Weights: 1/3 (rest), 1/18 (|c|=1), 1/36 (|c|=sqrt 2).  c_s^2 = 1/3 (Sec. II.C,
below the equation of state).
"""
import numpy as np

Q = 19

C = np.array([
    [0, 0, 0],
    [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
    [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1],
], dtype=np.int64)

W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)

OPP = np.array([int(np.where((C == -C[q]).all(axis=1))[0][0]) for q in range(Q)])

CS2 = 1.0 / 3.0

# unit vectors of the three axes (x, y, z)
AXES = np.eye(3, dtype=np.int64)


def shift(a, c):
    """Value of field ``a`` at x + c, returned at x (periodic).

    ``a`` is indexed [..., z, y, x]; ``c`` = (cx, cy, cz)."""
    cx, cy, cz = int(c[0]), int(c[1]), int(c[2])
    return np.roll(a, shift=(-cz, -cy, -cx), axis=(-3, -2, -1))


def place(a, c):
    """Move the value at x to x + c (periodic): inverse of ``shift``."""
    cx, cy, cz = int(c[0]), int(c[1]), int(c[2])
    return np.roll(a, shift=(cz, cy, cx), axis=(-3, -2, -1))


def equilibrium(rho, u):
    """Second-order equilibrium of Sec. II.A (equation below the discrete BGK
    equation): w_d rho [1 + c.u/cs2 + (c.u)^2/(2 cs4) - u.u/(2 cs2)].

    rho: (...), u: (3, ...).  Returns (19, ...)."""
    usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    out = np.empty((Q,) + rho.shape)
    for q in range(Q):
        cu = C[q, 0] * u[0] + C[q, 1] * u[1] + C[q, 2] * u[2]
        out[q] = W[q] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq / (2.0 * CS2))
    return out

"""Colloid forces and motion (Sec. II.E).  TEST INFRASTRUCTURE ONLY.

Total force on colloid j (Sec. II.E, Newton equation):
  * fluid: momentum exchanged on its bounce-back links during the step, plus
    the momentum of fluid it covers and minus the momentum of fluid it
    uncovers (node creation/deletion);
  * electric: sum over its surface nodes of q_c E (reading of the printed
    -Q grad phi for a charge carried by surface nodes);
  * Hertz contact (eq. colloid_interaction), k_H delta^{3/2} along the line of
    centres, repulsive (reading: the printed gradient sign would attract);
  * lubrication (eq. lubrication) for surface gaps 0 < h < 2/3, with
    eta = rho_ref c_s^2 (tau - 1/2), rho_ref = 1, and the printed bracket
    (1/h - 1).

Motion: velocity-Verlet with the force of the current step held over the
step: x(t+1) = x + v + F/(2m), v(t+1) = v + F/m, m = rho_p (4/3) pi r^3.

Remap after the move (Sec. II.E, projection figure and the two node-conversion
equations): a node covered by the colloid gives its fluid momentum to the
colloid, its populations are removed and its ions are spread equally over its
D3Q19 neighbours that are fluid both before and after the move (reading: a
neighbour uncovered in the same move starts with zero ions, so it receives
none and ions are conserved exactly); a node uncovered by the colloid is refilled with the
equilibrium at the mean density of its fluid neighbours and the colloid
velocity, the colloid loses that momentum, and its ions start at zero.
Reading: signs of the two momentum terms are those that conserve total
momentum; the refill velocity is the colloid velocity.
"""
import math

import numpy as np

from .geometry import min_image
from .lattice import C, CS2, Q, equilibrium, shift


def pair_forces(X, V, R, dims, k_hertz, eta):
    n = X.shape[0]
    F = np.zeros((n, 3))
    for i in range(n):
        for j in range(i + 1, n):
            d = np.array([min_image(X[i, a] - X[j, a], dims[a]) for a in range(3)])
            dist = float(np.sqrt((d * d).sum()))
            if dist == 0.0:
                continue
            nh = d / dist
            overlap = R[i] + R[j] - dist
            if overlap > 0.0:
                fh = k_hertz * overlap ** 1.5 * nh
                F[i] += fh
                F[j] -= fh
            gap = dist - (R[i] + R[j])
            if 0.0 < gap < 2.0 / 3.0:
                vrel = float(nh @ (V[i] - V[j]))
                fl = -1.5 * math.pi * eta * R[i] * R[j] * nh * vrel * (1.0 / gap - 1.0)
                F[i] += fl
                F[j] -= fl
    return F


def total_force(sys, E, p_bb):
    nc = sys.cx.shape[0]
    F = p_bb.copy()
    for j in range(nc):
        m = sys.surface & (sys.owner == j)
        for a in range(3):
            F[j, a] += float((sys.qc[m] * E[a][m]).sum())
    eta = 1.0 * CS2 * (sys.tau - 0.5)
    F += pair_forces(sys.cx, sys.cv, sys.cr, (sys.nx, sys.ny, sys.nz), sys.k_hertz, eta)
    return F


def move_and_remap(sys):
    F = sys.colloid_force
    m = sys.cmass[:, None]
    a = F / m
    X = sys.cx + sys.cv + 0.5 * a
    V = sys.cv + a
    dims = np.array([sys.nx, sys.ny, sys.nz], dtype=np.float64)
    X = np.where(X < 0.0, X + dims, X)
    X = np.where(X >= dims, X - dims, X)

    solid_old = sys.solid.copy()
    owner_old = sys.owner.copy()
    sys.cx = X
    sys._geometry()
    solid_new = sys.solid
    owner_new = sys.owner
    fluid_new = ~solid_new
    created = solid_new & ~solid_old
    deleted = ~solid_new & solid_old
    dV = np.zeros_like(V)

    # covered nodes: fluid momentum to the colloid, ions to fluid neighbours
    if created.any():
        mom = np.zeros((3,) + sys.shape)
        for q in range(1, Q):
            s = sys.f[:, q].sum(axis=0)
            for ax in range(3):
                if C[q, ax] != 0:
                    mom[ax] += C[q, ax] * s
        own = owner_new[created]
        for ax in range(3):
            np.add.at(dV[:, ax], own, mom[ax][created])
        if sys.nions:
            kept = fluid_new & ~solid_old  # fluid before and after the move
            cnt = np.zeros(sys.shape)
            for q in range(1, Q):
                cnt += shift(kept, C[q])
            share = np.where(created & (cnt > 0), 1.0 / np.maximum(cnt, 1.0), 0.0)
            add = np.zeros_like(sys.n)
            for q in range(1, Q):
                # node y = x + c_q receives from created node x
                for s in range(2):
                    add[s] += shift(sys.n[s] * share, -C[q]) * kept
            sys.n = (sys.n + add) * fluid_new
        sys.f[:, :, created] = 0.0

    # uncovered nodes: equilibrium refill at the neighbour-mean density
    if deleted.any():
        old_fluid = ~solid_old & fluid_new
        rho = sys.f.sum(axis=1) * old_fluid
        tot = np.zeros_like(rho)
        cnt = np.zeros(sys.shape)
        for q in range(1, Q):
            tot += shift(rho, C[q])
            cnt += shift(old_fluid, C[q])
        rbar = np.where(cnt > 0, tot / np.maximum(cnt, 1.0), 0.0)
        idx = np.argwhere(deleted)
        for (z, y, x) in idx:
            j = int(owner_old[z, y, x])
            vj = V[j]
            for s_ in range(sys.ncomp):
                r = rbar[s_, z, y, x]
                sys.f[s_, :, z, y, x] = equilibrium(np.array(r), vj)
                dV[j] -= r * vj
        if sys.nions:
            sys.n[:, deleted] = 0.0
    sys.cv = V + dV / m

"""A second, deliberately naive FP64 transcription of one coupled timestep
(Sec. II.A-E), written with explicit loops over lattice sites and directions
for tiny boxes.  Test helper only: it imports nothing from the oracle or the
product.  Its job is to catch transcription slips of the array-shift oracle
(a shifted index, a wrong neighbour direction, a dropped term) by an
implementation whose structure differs: every value is formed site by site
from the model equations, and the Poisson equation is solved by a dense
linear solve.

Model statements (and readings) follow the paper:
  * macro fields (Sec. II.A): rho^s = sum_q f^s_q, J = sum_s sum_q f^s_q c_q,
    virtual densities on interface solid nodes = mean over fluid D3Q19
    neighbours (Sec. II.E), psi = 1 - exp(-rho) (Sec. II.C), eps from the
    colour c and the solid fraction (Sec. II.B, II.E), q = n+ - n- + q_c;
  * Poisson (Sec. II.B): sum_d k_{i+d/2} (phi_{i+d} - phi_i) = -(q_i - qbar)
    + sum_d k_{i+d/2} (E_ext . c_d), k = mean of the two cell permittivities,
    mean(phi) = 0; field E = -(central difference of phi) + E_ext;
  * ion face flux through face (i, i+a) (Sec. II.B, II.E):
    D psi_f(i) psi_f(i+a) [dn~ - z nbar~ Ebar_a - (dmu/drho_a) nbar~ drho_a];
  * forces (Sec. II.C): Shan-Chen fluid-fluid and fluid-ion sums with the
    D3Q19 weights, friction -(1/D) half the flux through each face of a cell,
    Kelvin (eps_i - eps_bar)/4 sum_d |E(i+d)|^2 c_d, split over the
    components by rho^s / rho;
  * Nernst-Planck update with upwind push advection at the physical velocity
    (J + sum Phi / 2)/rho, no advective transfer across a face touching a
    solid node (Sec. II.B);
  * BGK collision at u + tau Phi^s / rho^s, pull of the post-collision values
    by the neighbours, halfway bounce-back with the moving-wall term
    6 w_q rho (c_q . v) (Sec. II.A, II.E).
"""
import math

import numpy as np

CV = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
      (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
      (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
WT = [1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12


def _opp(q):
    c = CV[q]
    return CV.index((-c[0], -c[1], -c[2]))


def _feq(rho, u, q):
    c = CV[q]
    cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
    uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    return WT[q] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)


class NaiveSystem:
    """State: f[s][q][z][y][x], n[s][z][y][x], phi; geometry arrays given."""

    def __init__(self, p, f, n, phi, solid, owner, psi_s, qc, cv):
        self.p = p
        self.nx, self.ny, self.nz = p.nx, p.ny, p.nz
        self.f = np.array(f, dtype=np.float64)
        self.n = np.array(n, dtype=np.float64)
        self.phi = np.array(phi, dtype=np.float64)
        self.solid = np.array(solid, dtype=bool)
        self.owner = np.array(owner)
        self.psi_s = np.array(psi_s, dtype=np.float64)
        self.qc = np.array(qc, dtype=np.float64)
        self.cv = np.array(cv, dtype=np.float64).reshape(-1, 3)
        er = 1.0 / (4.0 * math.pi * p.bjerrum)
        self.ea, self.eb, self.ep = p.eps_r[0] * er, p.eps_r[1] * er, p.eps_r_colloid * er

    def sites(self):
        for z in range(self.nz):
            for y in range(self.ny):
                for x in range(self.nx):
                    yield z, y, x

    def nb(self, z, y, x, c):
        return (z + c[2]) % self.nz, (y + c[1]) % self.ny, (x + c[0]) % self.nx

    def step(self):
        p = self.p
        nc = p.ncomp
        sh = (self.nz, self.ny, self.nx)
        fluid = ~self.solid
        # macro fields
        rho = np.zeros((nc,) + sh)
        J = np.zeros((3,) + sh)
        for s_ in self.sites():
            if not fluid[s_]:
                continue
            for s in range(nc):
                for q in range(19):
                    v = self.f[(s, q) + s_]
                    rho[(s,) + s_] += v
                    for a in range(3):
                        J[(a,) + s_] += v * CV[q][a]
        surface = np.zeros(sh, dtype=bool)
        for s_ in self.sites():
            if self.solid[s_]:
                surface[s_] = any(fluid[self.nb(*s_, CV[q])] for q in range(1, 19))
        rv = rho.copy()
        for s_ in self.sites():
            if surface[s_]:
                cnt = 0
                acc = [0.0] * nc
                for q in range(1, 19):
                    t = self.nb(*s_, CV[q])
                    if fluid[t]:
                        cnt += 1
                        for s in range(nc):
                            acc[s] += rho[(s,) + t]
                for s in range(nc):
                    rv[(s,) + s_] = acc[s] / cnt
        psi = -np.expm1(-rv)
        eps = np.zeros(sh)
        q_ = np.zeros(sh)
        for s_ in self.sites():
            ra = rv[(0,) + s_]
            rb = rv[(1,) + s_] if nc == 2 else 0.0
            c = (rb - ra) / (ra + rb) if ra + rb > 0 else 0.0
            ef = 0.5 * (self.ea * (1.0 - c) + self.eb * (1.0 + c))
            eps[s_] = self.psi_s[s_] * self.ep + (1.0 - self.psi_s[s_]) * ef
            q_[s_] = self.qc[s_] + (self.n[(0,) + s_] - self.n[(1,) + s_] if p.nions else 0.0)
        # Poisson: dense solve with the mean-zero constraint as an extra row
        N = self.nx * self.ny * self.nz
        idx = lambda z, y, x: (z * self.ny + y) * self.nx + x  # noqa: E731
        qbar = sum(q_[s_] for s_ in self.sites()) / N
        A = np.zeros((N + 1, N + 1))
        b = np.zeros(N + 1)
        for s_ in self.sites():
            i = idx(*s_)
            b[i] = -(q_[s_] - qbar)
            for q in range(1, 7):
                t = self.nb(*s_, CV[q])
                k = 0.5 * (eps[s_] + eps[t])
                A[i, idx(*t)] += k
                A[i, i] -= k
                b[i] += k * sum(p.E_ext[a] * CV[q][a] for a in range(3))
            A[i, N] = 1.0
            A[N, i] = 1.0
        sol = np.linalg.solve(A, b)
        phi = np.zeros(sh)
        for s_ in self.sites():
            phi[s_] = sol[idx(*s_)]
        self.phi = phi
        E = np.zeros((3,) + sh)
        for s_ in self.sites():
            for a in range(3):
                e = [0, 0, 0]
                e[a] = 1
                up = self.nb(*s_, e)
                dn = self.nb(*s_, (-e[0], -e[1], -e[2]))
                E[(a,) + s_] = -(phi[up] - phi[dn]) / 2.0 + p.E_ext[a]
        # ion face fluxes F[s][a] through the +a face of each cell
        psi_f = np.where(fluid, 1.0 - self.psi_s, 0.0)
        F = np.zeros((2, 3) + sh)
        if p.nions:
            for s_ in self.sites():
                for a in range(3):
                    e = [0, 0, 0]
                    e[a] = 1
                    t = self.nb(*s_, e)
                    w = psi_f[s_] * psi_f[t]
                    if w == 0.0:
                        continue
                    for s, z in ((0, 1.0), (1, -1.0)):
                        ni = self.n[(s,) + s_] / psi_f[s_]
                        nj = self.n[(s,) + t] / psi_f[t]
                        nbar = 0.5 * (ni + nj)
                        Eb = 0.5 * (E[(a,) + s_] + E[(a,) + t])
                        dr = rho[(0,) + t] - rho[(0,) + s_]
                        F[(s, a) + s_] = p.D * w * ((nj - ni) - z * nbar * Eb - (p.dmu[s] / p.drho_a) * nbar * dr)
        # forces
        Phi = np.zeros((nc, 3) + sh)
        ebar = 0.5 * (self.ea + self.eb)
        for s_ in self.sites():
            if not fluid[s_]:
                continue
            sc = np.zeros((nc, 3))
            fi = np.zeros(3)
            for q in range(1, 19):
                t = self.nb(*s_, CV[q])
                for a in range(3):
                    if nc == 2:
                        sc[0, a] += WT[q] * psi[(1,) + t] * CV[q][a]
                        sc[1, a] += WT[q] * psi[(0,) + t] * CV[q][a]
                    if p.nions:
                        for s in range(2):
                            if p.dmu[s] != 0.0:
                                fi[a] += (p.dmu[s] / (p.drho_a / 3.0)) * WT[q] * self.n[(s,) + t] * CV[q][a]
            fel = np.zeros(3)
            for a in range(3):
                e = [0, 0, 0]
                e[a] = 1
                up = self.nb(*s_, e)
                dn = self.nb(*s_, (-e[0], -e[1], -e[2]))
                E2u = sum(E[(b,) + up] ** 2 for b in range(3))
                E2d = sum(E[(b,) + dn] ** 2 for b in range(3))
                fel[a] += 0.25 * (eps[s_] - ebar) * (E2u - E2d)
                if p.nions:
                    tot = 0.0
                    for s in range(2):
                        tot += F[(s, a) + s_] + F[(s, a) + dn]
                    fel[a] += -tot / (2.0 * p.D)
            rt = sum(rho[(s,) + s_] for s in range(nc))
            for s in range(nc):
                for a in range(3):
                    v = 0.0
                    if nc == 2:
                        v += -p.G * psi[(s,) + s_] * sc[s, a]
                    if s == 0:
                        v += -psi[(0,) + s_] * fi[a]
                    v += (rho[(s,) + s_] / rt) * fel[a]
                    Phi[(s, a) + s_] = v
        u = np.zeros((3,) + sh)
        ub = np.zeros((3,) + sh)
        for s_ in self.sites():
            if not fluid[s_]:
                continue
            rt = sum(rho[(s,) + s_] for s in range(nc))
            for a in range(3):
                u[(a,) + s_] = (J[(a,) + s_] + 0.5 * sum(Phi[(s, a) + s_] for s in range(nc))) / rt
                ub[(a,) + s_] = J[(a,) + s_] / rt
        # Nernst-Planck update
        nn = self.n.copy()
        if p.nions:
            for s_ in self.sites():
                for a in range(3):
                    e = [0, 0, 0]
                    e[a] = 1
                    dn = self.nb(*s_, (-e[0], -e[1], -e[2]))
                    for s in range(2):
                        nn[(s,) + s_] += F[(s, a) + s_] - F[(s, a) + dn]
            for s_ in self.sites():
                if not fluid[s_]:
                    continue
                for q in range(1, 7):
                    t = self.nb(*s_, CV[q])
                    if not fluid[t]:
                        continue
                    ud = sum(u[(a,) + s_] * CV[q][a] for a in range(3))
                    if ud > 0.0:
                        for s in range(2):
                            amt = ud * self.n[(s,) + s_]
                            nn[(s,) + s_] -= amt
                            nn[(s,) + t] += amt
            nn[:, self.solid] = 0.0
        # collision, streaming, bounce-back
        fn = np.zeros_like(self.f)
        for s_ in self.sites():
            if not fluid[s_]:
                continue
            for s in range(nc):
                r = rho[(s,) + s_]
                ue = [ub[(a,) + s_] + (p.tau * Phi[(s, a) + s_] / r if r > 0 else 0.0) for a in range(3)]
                for q in range(19):
                    post = self.f[(s, q) + s_] + (_feq(r, ue, q) - self.f[(s, q) + s_]) / p.tau
                    t = self.nb(*s_, CV[q])
                    if fluid[t]:
                        fn[(s, q) + t] += post
                    else:
                        v = self.cv[self.owner[t]]
                        cvv = sum(CV[q][a] * v[a] for a in range(3))
                        fn[(s, _opp(q)) + s_] += post - 6.0 * WT[q] * r * cvv
        self.f = fn
        self.n = nn

"""One coupled lattice timestep of the electrohydrodynamic model (Sec. II).
TEST INFRASTRUCTURE ONLY.

State at time t: populations f^sigma_q(x) after streaming (pre-collision),
ion concentrations n^+-(x), the potential of the previous step (warm start of
the Poisson solve) and the colloid table.  Order of one step (the paper gives
none explicitly):

  1. macro fields: rho^sigma, momentum, virtual densities on interface solid
     nodes, pseudopotentials psi^sigma, permittivity eps, charge q;
  2. Poisson solve for phi (Sec. II.D);
  3. field E = -grad phi + E_ext (Sec. II.B);
  4. ion face fluxes on the D3Q7 faces (Sec. II.B, II.E);
  5. forces on the fluids: Shan-Chen fluid-fluid and fluid-ion, friction,
     Kelvin (Sec. II.C);
  6. Nernst-Planck update with upwind advection (Sec. II.B);
  7. forced BGK collision, streaming, halfway bounce-back with the moving-wall
     correction and momentum exchange (Sec. II.A, II.E);
  8. moving colloids: forces, velocity-Verlet, remap (Sec. II.E).

Pins: every part above has its own pin (exact moments and symbols, brute
force, closed forms, conservation); the composed step is checked against a
site-by-site transcription with a dense Poisson solve on tiny lattices, by
exact conservation of mass, ions and charge, momentum with moving colloids,
the Young-Laplace law across drop radii, the low-zeta electrophoretic
mobility and the O'Konski deformation of a dielectric drop.  No worked
example of the paper fixes the composed step's values.

Lattice units: dx = dt = e = beta = rho0 = 1.  sigma = 0 is component a
("red", water), sigma = 1 is component b ("blue", oil).  Species s = 0 is the
cation (z = +1), s = 1 the anion (z = -1).
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry, poisson
from .lattice import AXES, C, CS2, OPP, Q, W, equilibrium, place, shift


def psi_of(rho):
    """Pseudopotential psi = rho0 (1 - exp(-rho/rho0)), rho0 = 1 (Sec. II.C)."""
    return -np.expm1(-rho)


def virtual_density(rho, solid, surface):
    """Jansen correction (Sec. II.E, last paragraph before the projection
    figure): interface solid nodes carry the mean density of their fluid D3Q19
    neighbours.  Reading: the paper's printed sum is the mean it describes in
    words.  Other solid nodes keep 0.  rho: (ncomp, ...)."""
    fluid = ~solid
    out = rho * fluid
    s = np.zeros_like(rho)
    cnt = np.zeros(solid.shape)
    for q in range(1, Q):
        s += shift(rho * fluid, C[q])
        cnt += shift(fluid, C[q])
    mean = np.where(cnt > 0, s / np.maximum(cnt, 1.0), 0.0)
    return np.where(surface, mean, out)


def permittivity(rho_v, psi_s, eps_a, eps_b, eps_p):
    """eps = psi_s eps_p + (1 - psi_s) eps_f(c) (Sec. II.E last equation) with
    eps_f = [eps_a (1 - c) + eps_b (1 + c)] / 2, c = (rho_b - rho_a)/(rho_a + rho_b)
    (Sec. II.B eq. dielectric_constant); c = 0 where both densities vanish."""
    ra = rho_v[0]
    rb = rho_v[1] if rho_v.shape[0] > 1 else np.zeros_like(ra)
    tot = ra + rb
    c = np.where(tot > 0, (rb - ra) / np.where(tot > 0, tot, 1.0), 0.0)
    eps_f = 0.5 * (eps_a * (1.0 - c) + eps_b * (1.0 + c))
    return psi_s * eps_p + (1.0 - psi_s) * eps_f


def electric_field(phi, E_ext):
    """E = -grad phi_I + E_ext, central differences (Sec. II.B, potential split)."""
    E = np.empty((3,) + phi.shape)
    for a in range(3):
        e = AXES[a]
        E[a] = -(shift(phi, e) - shift(phi, -e)) / 2.0 + E_ext[a]
    return E


def face_fluxes(n, psi_f, E, rho_a, D, dmu, drho_a):
    """Ion fluxes through the three owned faces i + e_a/2 of every cell
    (Sec. II.B eq. ionic-fluxes-disc with the solid-fraction weighting of
    Sec. II.E eq. ionic-fluxes-disc-2).

    Returns F[s, a] = j^s_{i+a/2} . c_a, the amount entering cell i through its
    +a face per step, in the convention of eq. ionic-fluxes-disc (j = D grad n
    + ...; n(t+1) = n + sum_d j.c_d).  With n~ = n/psi_f and z = +-1:

      F = D psi_f(i) psi_f(i+a) [ (n~_{i+a} - n~_i)
            - z (n~_i + n~_{i+a})/2 (E_a(i) + E_a(i+a))/2
            - (dmu/drho_a) (n~_i + n~_{i+a})/2 (rho_a(i+a) - rho_a(i)) ].

    Readings: the two printed forms differ by an overall sign; the convention
    of eq. ionic-fluxes-disc is kept, which makes sum_d j.c_d the discrete
    Laplacian.  E(r'_i) is read as E(r_{i+d}).  The solvation sign follows the
    equilibrium n ∝ exp(-z phi - mu_s) with mu_s = -(dmu/drho_a) rho_a
    (Sec. II.C eq. solvation_potential and Sec. III.A), which gives
    n_b/n_a = exp(-dmu)."""
    ns = n.shape[0]
    ntil = np.where(psi_f > 0, n / np.where(psi_f > 0, psi_f, 1.0), 0.0)
    F = np.zeros((ns, 3) + psi_f.shape)
    zval = (1.0, -1.0)
    for a in range(3):
        e = AXES[a]
        pf = psi_f * shift(psi_f, e)
        Ebar = 0.5 * (E[a] + shift(E[a], e))
        drho = shift(rho_a, e) - rho_a
        for s in range(ns):
            ni = ntil[s]
            nj = shift(ntil[s], e)
            nbar = 0.5 * (ni + nj)
            F[s, a] = D * pf * ((nj - ni) - zval[s] * nbar * Ebar - (dmu[s] / drho_a) * nbar * drho)
    return F


def np_update(n, F, u, fluid):
    """Finite-volume Nernst-Planck update on the D3Q7 faces (Sec. II.B eq.
    nernst-planck-disc) with first-order upwind advection.

    Reading (the printed advective sum uses only u(r_i), n(r_i) and so only
    removes ions): each cell sends H(u_i.c_d)(u_i.c_d) n_i to its neighbour
    i + d and the neighbour receives the same amount (push form), so ions are
    conserved exactly.  No advective transfer crosses a face with a solid node
    on either side.  u is the physical fluid velocity."""
    out = n.copy()
    for s in range(n.shape[0]):
        div = np.zeros_like(n[s])
        for a in range(3):
            div += F[s, a] - shift(F[s, a], -AXES[a])
        adv_out = np.zeros_like(n[s])
        adv_in = np.zeros_like(n[s])
        for a in range(3):
            for sign in (1, -1):
                cd = sign * AXES[a]
                ud = sign * u[a]
                amt = np.maximum(ud, 0.0) * n[s] * (fluid & shift(fluid, cd))
                adv_out += amt
                adv_in += place(amt, cd)
        out[s] = n[s] + div - adv_out + adv_in
    return out


def shan_chen_sum(field):
    """sum_{d=1..18} w_d field(x + c_d) c_d  (Sec. II.C eq. shanChenForce)."""
    out = np.zeros((3,) + field.shape)
    for q in range(1, Q):
        v = W[q] * shift(field, C[q])
        for a in range(3):
            if C[q, a] != 0:
                out[a] += C[q, a] * v
    return out


def friction_force(F, D):
    """F_fr(i) = -(1/(beta D)) sum_s (1/2) sum_{d in Q6} (j^s_{i+d/2}.c_d) c_d
    (Sec. II.C eq. frictionforce, discretised on the faces).  Reading: the
    factor 1/2 shares every face between its two cells, so that the total
    force equals -(1/(beta D)) times the sum of all face fluxes; the printed
    per-cell sum counts each face twice."""
    out = np.zeros((3,) + F.shape[2:])
    for a in range(3):
        tot = np.zeros(F.shape[2:])
        for s in range(F.shape[0]):
            tot += F[s, a] + shift(F[s, a], -AXES[a])
        out[a] = -tot / (2.0 * D)
    return out


def kelvin_force(eps, eps_bar, E):
    """Kelvin (dielectric) force F_K = +(1/2)(eps - eps_bar) grad |E|^2 by
    central differences, i.e. (eps_i - eps_bar)/4 sum_{d in Q6} |E(i+d)|^2 c_d
    (Sec. II.C, discrete total-force equation).

    Reading: the continuum eq. kelvin prints a minus sign, the discrete form a
    plus.  The plus sign is the one that follows from the cited Korteweg-
    Helmholtz density -E^2 grad(eps)/2 + grad(E^2 c deps/dc)/2 with the linear
    eps(c) of eq. dielectric_constant, and the only one under which an
    ion-free drop elongates along the applied field as Sec. III.B reports
    (the minus sign flattens it)."""
    E2 = E[0] * E[0] + E[1] * E[1] + E[2] * E[2]
    out = np.empty((3,) + eps.shape)
    for a in range(3):
        out[a] = 0.25 * (eps - eps_bar) * (shift(E2, AXES[a]) - shift(E2, -AXES[a]))
    return out


class OracleSystem:
    """State and timestep of one periodic lattice system."""

    def __init__(self, params, rho, n=None, u=None, colloid_x=None, colloid_v=None,
                 colloid_q=None, colloid_r=None, phi=None):
        p = params
        self.p = p
        self.nx, self.ny, self.nz = int(p.nx), int(p.ny), int(p.nz)
        self.shape = (self.nz, self.ny, self.nx)
        self.ncomp = int(p.ncomp)
        self.nions = int(p.nions)
        self.tau = float(p.tau)
        self.G = float(p.G)
        self.D = float(p.D)
        eps_ref = 1.0 / (4.0 * math.pi * float(p.bjerrum))
        self.eps_a = float(p.eps_r[0]) * eps_ref
        self.eps_b = float(p.eps_r[1]) * eps_ref
        self.eps_p = float(p.eps_r_colloid) * eps_ref
        self.eps_bar = 0.5 * (self.eps_a + self.eps_b)
        self.dmu = (float(p.dmu[0]), float(p.dmu[1]))
        self.drho_a = float(p.drho_a)
        self.E_ext = tuple(float(v) for v in p.E_ext)
        self.tol = float(p.poisson_tol)
        self.max_iter = int(p.poisson_max_iter)
        self.h = int(p.psi_subdiv)
        self.moving = bool(p.colloids_move)
        self.rho_p = float(p.rho_p)
        self.k_hertz = float(p.k_hertz)

        rho = np.asarray(rho, dtype=np.float64).reshape((self.ncomp,) + self.shape)
        self.cx = np.zeros((0, 3)) if colloid_x is None else np.array(colloid_x, dtype=np.float64).reshape(-1, 3)
        nc = self.cx.shape[0]
        self.cv = np.zeros((nc, 3)) if colloid_v is None else np.array(colloid_v, dtype=np.float64).reshape(-1, 3)
        self.cq = np.zeros(nc) if colloid_q is None else np.array(colloid_q, dtype=np.float64).reshape(-1)
        self.cr = np.zeros(nc) if colloid_r is None else np.array(colloid_r, dtype=np.float64).reshape(-1)
        self.cmass = self.rho_p * (4.0 / 3.0) * math.pi * self.cr ** 3
        self._geometry()

        uu = np.zeros((3,) + self.shape) if u is None else np.asarray(u, dtype=np.float64)
        self.f = np.stack([equilibrium(rho[s], uu) for s in range(self.ncomp)])
        self.f *= self.fluid  # no fluid on solid nodes
        if self.nions:
            self.n = np.asarray(n, dtype=np.float64).reshape((2,) + self.shape) * self.fluid
        else:
            self.n = np.zeros((0,) + self.shape)
        self.phi = np.zeros(self.shape) if phi is None else np.asarray(phi, dtype=np.float64).copy()
        self.t = 0
        self.poisson_iters = 0
        self.poisson_relres = 0.0
        self.colloid_force = np.zeros((nc, 3))

    # ---------------------------------------------------------------- geometry
    def _geometry(self):
        nc = self.cx.shape[0]
        if nc:
            self.solid, self.owner, self.psi_s = geometry.project(
                self.nx, self.ny, self.nz, self.cx, self.cr, self.h)
        else:
            self.solid = np.zeros(self.shape, dtype=bool)
            self.owner = np.full(self.shape, -1, dtype=np.int64)
            self.psi_s = np.zeros(self.shape)
        self.fluid = ~self.solid
        self.surface = geometry.surface_nodes(self.solid)
        self.psi_f = np.where(self.fluid, 1.0 - self.psi_s, 0.0)
        self.qc = geometry.colloid_charge(self.owner, self.surface, self.cq)

    # ----------------------------------------------------------- macro fields
    def macro(self):
        """rho^sigma, momentum J, virtual densities, psi, eps, q at time t."""
        fl = self.fluid
        rho = self.f.sum(axis=1) * fl
        J = np.zeros((3,) + self.shape)
        for q in range(1, Q):
            s = self.f[:, q].sum(axis=0)
            for a in range(3):
                if C[q, a] != 0:
                    J[a] += C[q, a] * s
        J *= fl
        rho_v = virtual_density(rho, self.solid, self.surface)
        psi = psi_of(rho_v)
        eps = permittivity(rho_v, self.psi_s, self.eps_a, self.eps_b, self.eps_p)
        q = self.qc.copy()
        if self.nions:
            q += self.n[0] - self.n[1]
        return rho, J, rho_v, psi, eps, q

    # ------------------------------------------------------------------ step
    def step(self):
        fl = self.fluid
        rho, J, rho_v, psi, eps, q = self.macro()
        self.last_rho_v, self.last_eps, self.last_q = rho_v, eps, q

        # 2-3. potential and field
        if self.nions or self.qc.any() or any(self.E_ext):
            self.phi, self.poisson_iters, self.poisson_relres = poisson.solve(
                q, eps, self.phi, self.tol, self.max_iter, self.E_ext)
        E = electric_field(self.phi, self.E_ext)
        self.last_E = E

        # 4. ion face fluxes
        if self.nions:
            F = face_fluxes(self.n, self.psi_f, E, rho[0], self.D, self.dmu, self.drho_a)
        else:
            F = np.zeros((0, 3) + self.shape)

        # 5. forces on the fluid components
        Phi = np.zeros((self.ncomp, 3) + self.shape)
        if self.ncomp == 2 and self.G != 0.0:
            Phi[0] += -self.G * psi[0] * shan_chen_sum(psi[1])
            Phi[1] += -self.G * psi[1] * shan_chen_sum(psi[0])
        if self.nions and (self.dmu[0] != 0.0 or self.dmu[1] != 0.0):
            acc = np.zeros((3,) + self.shape)
            for s in range(2):
                if self.dmu[s] != 0.0:
                    G_as = self.dmu[s] / (self.drho_a * CS2)
                    acc += G_as * shan_chen_sum(self.n[s])
            Phi[0] += -psi[0] * acc
        Fel = kelvin_force(eps, self.eps_bar, E)
        if self.nions:
            Fel = Fel + friction_force(F, self.D)
        rho_tot = rho.sum(axis=0)
        safe = np.where(rho_tot > 0, rho_tot, 1.0)
        for s in range(self.ncomp):
            Phi[s] += (rho[s] / safe) * Fel
        Phi *= fl
        u_phys = (J + 0.5 * Phi.sum(axis=0)) / safe * fl
        u_bar = J / safe * fl
        self.last_u = u_phys
        self.last_Phi = Phi

        # 6. Nernst-Planck
        if self.nions:
            n_new = np_update(self.n, F, u_phys, fl)
        else:
            n_new = self.n

        # 7. collision, streaming, bounce-back
        fnew = np.zeros_like(self.f)
        nc = self.cx.shape[0]
        p_bb = np.zeros((nc, 3))
        for s in range(self.ncomp):
            rs = np.where(rho[s] > 0, rho[s], 1.0)
            ue = np.where(rho[s] > 0, u_bar + self.tau * Phi[s] / rs, u_bar)
            feq = equilibrium(rho[s], ue)
            fpost = self.f[s] + (feq - self.f[s]) / self.tau
            for qd in range(Q):
                c = C[qd]
                src = fpost[qd] * fl
                dest_fluid = shift(fl, c)
                fnew[s, qd] += place(src * dest_fluid, c)
                if nc:
                    bb = fl & ~dest_fluid
                    if bb.any():
                        own = shift(self.owner, c)[bb]
                        cv = self.cv[own] @ c.astype(np.float64)
                        val = fpost[qd][bb] - 6.0 * W[qd] * rho[s][bb] * cv
                        fnew[s, OPP[qd]][bb] += val
                        dp = (2.0 * fpost[qd][bb] - 6.0 * W[qd] * rho[s][bb] * cv)
                        for a in range(3):
                            if c[a] != 0:
                                np.add.at(p_bb[:, a], own, c[a] * dp)
        fnew *= fl
        self.f = fnew
        self.n = n_new * fl if self.nions else n_new

        # 8. colloids
        self.p_bb = p_bb
        if nc:
            from . import colloids
            self.colloid_force = colloids.total_force(self, E, p_bb)
            if self.moving:
                colloids.move_and_remap(self)
        self.t += 1

    def run(self, nsteps):
        for _ in range(int(nsteps)):
            self.step()

    # --------------------------------------------------------- read-outs
    def densities(self):
        return self.f.sum(axis=1) * self.fluid

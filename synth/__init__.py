"""Seeded synthetic inputs for the coupled electrohydrodynamic lattice step.

This module only draws initial conditions and parameter sets: density slabs and
droplets with seeded noise, uniform salt, colloid positions and charges.  It holds
none of the method's arithmetic (no equilibria, forces, fluxes, geometry
projection or Poisson solve), so both the CUDA path and the CPU oracle can read
its output without sharing any part of the model.

Arrays are float64, indexed [z, y, x] (x fastest), the layout of the library.
Lattice units throughout: dx = dt = e = beta = rho0 = 1.

Workloads follow the model of Rivas et al. (arXiv:1712.08494, Sec. II) and the
test geometries of its Sec. III (flat interfaces, droplets, suspensions).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import Dict, List, Optional

import numpy as np


@dataclass
class Params:
    """Parameter set of one lattice system (mirrors ``lbeh_params`` in lbeh.h)."""

    nx: int
    ny: int
    nz: int
    ncomp: int = 2
    nions: int = 2
    prec: str = "fp32"  # fp64 | fp32 | bf16 | fp16 (storage of populations)
    tau: float = 1.0
    G: float = 4.0
    rho0_shift: tuple = (0.0, 0.0)
    D: float = 0.05
    bjerrum: float = 0.4
    eps_r: tuple = (1.0, 0.5)
    eps_r_colloid: float = 0.125
    dmu: tuple = (0.0, 0.0)
    drho_a: float = 0.66
    E_ext: tuple = (0.0, 0.0, 0.0)
    poisson_tol: float = 1e-6
    poisson_max_iter: int = 50
    ncolloid_max: int = 0
    rho_p: float = 5.0
    k_hertz: float = 1.0
    psi_subdiv: int = 3
    colloids_move: int = 0
    poisson_solver: str = "auto"  # auto | multigrid | spectral

    def as_dict(self) -> dict:
        return asdict(self)


@dataclass
class Workload:
    """A parameter set plus the initial fields of one system."""

    name: str
    params: Params
    rho: np.ndarray            # (ncomp, nz, ny, nx)
    n: Optional[np.ndarray]    # (2, nz, ny, nx) cation/anion concentration, or None
    colloid_x: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))  # (N,3) x,y,z
    colloid_v: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    colloid_q: np.ndarray = field(default_factory=lambda: np.zeros((0,)))
    colloid_r: np.ndarray = field(default_factory=lambda: np.zeros((0,)))
    steps: int = 1
    note: str = ""
    u: Optional[np.ndarray] = None  # (3, nz, ny, nx) initial velocity, or None for rest

    @property
    def nsites(self) -> int:
        p = self.params
        return p.nx * p.ny * p.nz


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def _noise(rng, shape, amp):
    return 1.0 + rng.uniform(-amp, amp, size=shape)


def _far_mask(nx, ny, nz, centres, radii, margin):
    """Nodes farther than r+margin (minimum image) from every sphere centre.

    Used only to place neutralising counter-ions where no colloid can ever
    cover them; it is not the method's solid projection."""
    x, y, z = _grid(nx, ny, nz)
    far = np.ones((nz, ny, nx), dtype=bool)
    for (cx, cy, cz), r in zip(centres, radii):
        dx = np.abs(x - cx); dx = np.minimum(dx, nx - dx)
        dy = np.abs(y - cy); dy = np.minimum(dy, ny - dy)
        dz = np.abs(z - cz); dz = np.minimum(dz, nz - dz)
        far &= (dx * dx + dy * dy + dz * dz) > (r + margin) ** 2
    return far


def two_slab(nx=32, ny=32, nz=32, seed=0, G=0.08, prec="fp64", colloid=True,
             tol=1e-10, steps=200, noise=0.01) -> Workload:
    """Plain-method case: two flat interfaces (red 0.7/blue 0.04 for z<nz/2,
    swapped above), +-1% seeded density noise, salt 0.01, one fixed sphere of
    radius 4 centred at (16, 16, 15.5) with charge -20 e on its surface.

    Counter-cations (+20 e) are spread uniformly over nodes more than r+2 from
    the sphere so that the periodic system is neutral."""
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    x, y, z = _grid(nx, ny, nz)
    lower = z < nz // 2
    red = np.where(lower, 0.7, 0.04) * _noise(rng, shape, noise)
    blue = np.where(lower, 0.04, 0.7) * _noise(rng, shape, noise)
    rho = np.stack([red, blue])
    n = np.full((2,) + shape, 0.01)
    cx = np.zeros((0, 3)); cq = np.zeros(0); cr = np.zeros(0)
    if colloid:
        cx = np.array([[nx / 2.0, ny / 2.0, nz / 2.0 - 0.5]])
        cq = np.array([-20.0]); cr = np.array([4.0])
        far = _far_mask(nx, ny, nz, cx, cr, 2.0)
        n[0][far] += 20.0 / far.sum()
    p = Params(nx=nx, ny=ny, nz=nz, ncomp=2, nions=2, prec=prec, tau=1.0, G=G,
               D=0.05, bjerrum=0.4, eps_r=(1.0, 0.5), eps_r_colloid=0.125,
               dmu=(0.0, 0.0), drho_a=0.66, E_ext=(0.0, 0.0, 0.0),
               poisson_tol=tol, poisson_max_iter=200,
               ncolloid_max=len(cr), colloids_move=0)
    return Workload("two_slab_%d" % nx, p, rho, n, cx, np.zeros_like(cx), cq, cr, steps,
                    "flat interfaces + fixed charged sphere")


def droplet(n=128, r=24.0, seed=1, G=4.0, prec="fp32", salt=1e-3, Ez=1e-3, eps_r=(1.0, 0.5),
            charge=0.0, tol=1e-6, steps=5000, noise=0.01, nions=2) -> Workload:
    """Blue droplet of radius r at the box centre in red (0.7/0.04 swapped
    inside), +-1% seeded noise, uniform salt, applied field along z.

    A net droplet charge Q is carried by Q/V_in extra cations inside the drop
    and Q/V_out extra anions outside, which keeps the box neutral."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    x, y, z = _grid(n, n, n)
    c = n / 2.0
    inside = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 < r * r
    red = np.where(inside, 0.04, 0.7) * _noise(rng, shape, noise)
    blue = np.where(inside, 0.7, 0.04) * _noise(rng, shape, noise)
    rho = np.stack([red, blue])
    ions = None
    if nions:
        ions = np.full((2,) + shape, float(salt))
        if charge != 0.0:
            ions[0][inside] += charge / inside.sum()
            ions[1][~inside] += charge / (~inside).sum()
    p = Params(nx=n, ny=n, nz=n, ncomp=2, nions=nions, prec=prec, tau=1.0, G=G,
               D=0.05, bjerrum=0.4, eps_r=tuple(eps_r), eps_r_colloid=0.125,
               dmu=(0.0, 0.0), drho_a=0.66, E_ext=(0.0, 0.0, Ez),
               poisson_tol=tol, poisson_max_iter=50, ncolloid_max=0,
               rho0_shift=(0.04, 0.04))
    return Workload("droplet_%d" % n, p, rho, ions, steps=steps,
                    note="dielectric droplet r=%g, E_z=%g" % (r, Ez))


def suspension(n=256, ncoll=200, r=6.0, seed=2, prec="fp32", salt=1e-3, Ex=1e-3,
               qrange=(-40.0, -10.0), gap=2.0, tol=1e-6, steps=2000) -> Workload:
    """Single majority fluid (rho=1) with salt, ncoll non-overlapping spheres at
    seeded random positions (minimum surface gap `gap`), charges uniform in
    qrange, applied field along x.  Counter-cations neutralise the colloid
    charge, spread over nodes more than r+2 from every sphere."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    centres: List[np.ndarray] = []
    tries = 0
    while len(centres) < ncoll:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place colloids")
        p = rng.uniform(0.0, float(n), size=3)
        ok = True
        for c in centres:
            d = np.abs(p - c)
            d = np.minimum(d, n - d)
            if float(np.sqrt((d * d).sum())) < 2 * r + gap:
                ok = False
                break
        if ok:
            centres.append(p)
    cx = np.array(centres).reshape(-1, 3)
    cq = rng.uniform(qrange[0], qrange[1], size=ncoll)
    cr = np.full(ncoll, float(r))
    rho = np.ones((1,) + shape)
    ions = np.full((2,) + shape, float(salt))
    far = _far_mask(n, n, n, cx, cr, 2.0)
    ions[0][far] += -cq.sum() / far.sum()
    p = Params(nx=n, ny=n, nz=n, ncomp=1, nions=2, prec=prec, tau=1.0, G=0.0,
               D=0.05, bjerrum=0.4, eps_r=(1.0, 1.0), eps_r_colloid=0.125,
               dmu=(0.0, 0.0), drho_a=0.66, E_ext=(Ex, 0.0, 0.0),
               poisson_tol=tol, poisson_max_iter=50, ncolloid_max=ncoll,
               colloids_move=1, rho0_shift=(1.0, 0.0))
    return Workload("suspension_%d" % n, p, rho, ions, cx, np.zeros_like(cx), cq, cr, steps,
                    "moving charged spheres under an applied field")


def batch_boxes(nbox=96, seed=3, edges=(32, 40, 48, 56, 64), steps=1000) -> List[Workload]:
    """Independent charged droplets of uneven box size: edge drawn from
    `edges`, drop radius 0.3*edge, net charge U[0,200] e, E_z U[0,2e-3]."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(nbox):
        e = int(rng.choice(edges))
        q = float(rng.uniform(0.0, 200.0))
        ez = float(rng.uniform(0.0, 2e-3))
        w = droplet(n=e, r=0.3 * e, seed=1000 + b, charge=q, Ez=ez, steps=steps)
        w.name = "box%02d_%d" % (b, e)
        out.append(w)
    return out


def flat_interface(nx=512, ny=4, nz=4, dmu=(2.0, -2.0), chi=0.0, salt=1e-3, G=4.0, drho_a=0.66,
                   prec="fp32", tol=1e-8, D=0.05, nions=2, rho_major=0.7, rho_minor=0.04) -> Workload:
    """Quasi-one-dimensional box with two flat fluid interfaces (Sec. III.A):
    red (fluid a) rho_major/rho_minor (default 0.7/0.04) for x < nx/2,
    swapped for x >= nx/2, so the
    periodic box has interfaces near x = nx/2 and x = 0.  Permittivities
    eps_r = (1, (1 - chi)/(1 + chi)) give the contrast chi = (eps_a - eps_b) /
    (eps_a + eps_b).  Gibbs transfer energies dmu = (dmu+, dmu-); the initial
    salt is `salt` in fluid a and salt * exp(-(dmu+ + dmu-)/2) in fluid b, as
    the paper sets it.  No noise: the state is a function of x only."""
    shape = (nz, ny, nx)
    x, y, z = _grid(nx, ny, nz)
    in_a = x < nx // 2
    red = np.where(in_a, rho_major, rho_minor)
    blue = np.where(in_a, rho_minor, rho_major)
    rho = np.stack([red, blue])
    ions = None
    if nions:
        nb = salt * math.exp(-0.5 * (dmu[0] + dmu[1]))
        ions = np.stack([np.where(in_a, salt, nb)] * 2).astype(np.float64)
    p = Params(nx=nx, ny=ny, nz=nz, ncomp=2, nions=nions, prec=prec, tau=1.0, G=G,
               D=D, bjerrum=0.4, eps_r=(1.0, (1.0 - chi) / (1.0 + chi)), eps_r_colloid=0.125,
               dmu=tuple(float(v) for v in dmu), drho_a=float(drho_a), E_ext=(0.0, 0.0, 0.0),
               poisson_tol=tol, poisson_max_iter=200, ncolloid_max=0, rho0_shift=(0.04, 0.04))
    return Workload("flat_interface_%d" % nx, p, rho, ions, steps=1,
                    note="flat interfaces, dmu=%s, chi=%g" % (tuple(dmu), chi))


def interface_colloid(n=64, r=8.0, dz=0.0, salt=0.0, dmu=(4.0, 4.0), q=0.0, G=4.0, prec="fp32",
                      rho_major=0.7, rho_minor=0.04, tol=1e-6) -> Workload:
    """A sphere at a flat fluid interface (Sec. III.F): fluid a (red) for
    z < n/2, fluid b above (interfaces at z = n/2 - 1/2 and at the periodic
    boundary), one moving sphere of radius r centred dz above the middle
    interface with charge q, colloid permittivity 10/80 of the fluids'.  With
    salt > 0 the ions start at the bulk Boltzmann ratio of their Gibbs transfer
    energies, salt in fluid a and salt exp(-dmu) in fluid b; counter-ions
    for q are spread over nodes more than r + 2 from the sphere."""
    shape = (n, n, n)
    x, y, z = _grid(n, n, n)
    in_a = z < n // 2
    red = np.where(in_a, rho_major, rho_minor)
    blue = np.where(in_a, rho_minor, rho_major)
    rho = np.stack([red, blue])
    cx = np.array([[n / 2.0 + 0.25, n / 2.0 - 0.25, n / 2.0 - 0.5 + dz]])
    cr = np.array([float(r)])
    cq = np.array([float(q)])
    nions = 2 if (salt > 0.0 or q != 0.0) else 0
    ions = None
    if nions:
        ions = np.stack([np.where(in_a, salt, salt * math.exp(-dmu[0])),
                         np.where(in_a, salt, salt * math.exp(-dmu[1]))]).astype(np.float64)
        if q != 0.0:
            far = _far_mask(n, n, n, cx, cr, 2.0)
            ions[0 if q < 0 else 1][far] += abs(q) / far.sum()
    p = Params(nx=n, ny=n, nz=n, ncomp=2, nions=nions, prec=prec, tau=1.0, G=G, D=0.05, bjerrum=0.4,
               eps_r=(1.0, 1.0), eps_r_colloid=0.125, dmu=tuple(float(v) for v in dmu) if nions else (0.0, 0.0),
               drho_a=rho_major - rho_minor, E_ext=(0.0, 0.0, 0.0), poisson_tol=tol, poisson_max_iter=200,
               ncolloid_max=1, colloids_move=1, rho0_shift=(rho_minor, rho_minor))
    return Workload("interface_colloid_%d" % n, p, rho, ions, cx, np.zeros_like(cx), cq, cr, steps=1,
                    note="sphere r=%g at a flat interface, dz=%g, salt=%g" % (r, dz, salt))


def coated_droplet(n=128, rd=32.0, ncoll=80, rp=5.0, seed=5, prec="fp32", salt=1e-3, dmu=(4.0, -4.0), Ez=1e-3,
                   G=4.0, tol=1e-6, steps=2000) -> Workload:
    """Colloid-coated droplet (Sec. III.G): a drop of radius rd (fluid b) at
    the box centre, as the charged drop of Sec. III.D (uniform salt, Gibbs
    transfer energies dmu, equal fluid permittivities, field along z), with ncoll
    uncharged moving spheres of radius rp centred on the drop surface at the
    points of a Fibonacci lattice on the sphere (a homogeneous coating:
    covering fraction ncoll rp^2 / (4 rd^2)), particle permittivity 10/80 of
    the fluids', neutral wetting (interface solid nodes take the mean density
    of their fluid neighbours)."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    x, y, z = _grid(n, n, n)
    c = n / 2.0
    inside = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 < rd * rd
    red = np.where(inside, 0.04, 0.7) * _noise(rng, shape, 0.01)
    blue = np.where(inside, 0.7, 0.04) * _noise(rng, shape, 0.01)
    rho = np.stack([red, blue])
    k = np.arange(ncoll) + 0.5
    polar = np.arccos(1.0 - 2.0 * k / ncoll)
    azim = math.pi * (1.0 + math.sqrt(5.0)) * k
    cx = c + rd * np.stack([np.cos(azim) * np.sin(polar), np.sin(azim) * np.sin(polar), np.cos(polar)], axis=1)
    cr = np.full(ncoll, float(rp))
    ions = np.full((2,) + shape, float(salt))  # uniform: the transfer energies charge the drop over time
    p = Params(nx=n, ny=n, nz=n, ncomp=2, nions=2, prec=prec, tau=1.0, G=G, D=0.05, bjerrum=0.4,
               eps_r=(1.0, 1.0), eps_r_colloid=0.125, dmu=tuple(float(v) for v in dmu), drho_a=0.66,
               E_ext=(0.0, 0.0, Ez), poisson_tol=tol, poisson_max_iter=50, ncolloid_max=ncoll, colloids_move=1,
               rho0_shift=(0.04, 0.04))
    return Workload("coated_droplet_%d" % n, p, rho, ions, cx, np.zeros_like(cx), np.zeros(ncoll), cr, steps,
                    "drop r=%g coated by %d spheres r=%g, E_z=%g" % (rd, ncoll, rp, Ez))


def shear_wave(n=32, U=1e-3, rho=1.0, tau=1.0) -> Workload:
    """Single-component, ion-free periodic box whose initial velocity is the
    shear wave u_x(z) = U sin(2 pi z / n) (density uniform)."""
    shape = (n, n, n)
    p = Params(nx=n, ny=n, nz=n, ncomp=1, nions=0, prec="fp64", tau=tau, G=0.0)
    x, y, z = _grid(n, n, n)
    u = np.zeros((3,) + shape)
    u[0] = U * np.sin(2.0 * math.pi * z / n)
    return Workload("shear_wave_%d" % n, p, np.full((1,) + shape, rho), None, steps=1, u=u)


CONFIGS: Dict[str, callable] = {
    "two_slab": two_slab,
    "droplet": droplet,
    "suspension": suspension,
}

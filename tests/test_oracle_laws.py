"""Physical laws the composed oracle step must obey (CPU, slow).

* Young-Laplace (Sec. II.C eq. eqofstate, Sec. III.B): relaxed quasi-2D drops
  of several radii have a pressure jump, from the Shan-Chen equation of state
  p = c_s^2 (rho_a + rho_b) + c_s^2 G psi_a psi_b, that is linear in 1/R
  through zero, dp = gamma / R.  A drop radius is the radius of the disc whose
  area is the integral of the colour field c = (rho_b - rho_a)/(rho_a + rho_b)
  scaled from its outside to its inside value (the sharp-interface equivalent
  of the paper's c = 0 contour).  The slope is the surface tension; it agrees with the value
  measured on one drop by the script of tests/golden.
* Low-zeta electrophoresis (Sec. III.E): a weakly charged sphere
  (zeta = Q l_B / a = 0.27 kT/e) in a box whose only ions are its uniformly
  spread counter-ions is the kappa a -> 0 (Hueckel) limit.  The counter-ions
  carry the opposite force into the fluid as a uniform body force, so the
  sphere's velocity relative to the fluid is the settling velocity of a
  periodic array of spheres under the force Q E: mu = Q / (6 pi eta a K) with
  Hasimoto's periodic drag factor 1/K = 1 - 1.7601 phi^{1/3} + phi
  - 1.5593 phi^2 + 3.9799 phi^{8/3} - 3.0734 phi^{10/3} (phi: solid
  fraction).  The sphere is held fixed; the fluid flows past it at minus the
  mobility times E (relative motion is frame independent), and its steady
  mean velocity is extrapolated from the exponential approach of the last
  three samples.  Tolerance 15%: the hydrodynamic radius of a bounce-back
  sphere of radius 3 differs from 3 by a fraction of a lattice spacing.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import OracleSystem
from oracle.model import psi_of

HERE = os.path.dirname(os.path.abspath(__file__))


def _relaxed_drop(n, r, G, steps):
    w = synth.droplet(n=n, r=r, G=G, Ez=0.0, nions=0, tol=1e-8, noise=0.0)
    w.params.nx = 2
    rho = w.rho[:, :, :, n // 2 - 1:n // 2 + 1].copy()
    s = OracleSystem(w.params, rho)
    s.run(steps)
    ra, rb = s.densities()
    p = (ra + rb) / 3.0 + G / 3.0 * psi_of(ra) * psi_of(rb)
    c = n // 2
    dp = float(p[c, c, 0] - p[0, 0, 0])
    cc = ((rb - ra) / (rb + ra))[:, :, 0]
    c_in, c_out = float(cc[c, c]), float(cc[0, 0])
    area = float(((cc - c_out) / (c_in - c_out)).sum())
    return dp, math.sqrt(area / math.pi)


@pytest.mark.slow
def test_laplace_pressure_is_linear_in_inverse_radius():
    n, G = 48, 4.0
    pts = [_relaxed_drop(n, r, G, 2500) for r in (6.0, 10.0, 15.0)]
    dp = np.array([a for a, _ in pts])
    R = np.array([b for _, b in pts])
    A = np.stack([1.0 / R, np.ones_like(R)], axis=1)
    (gamma, c0), *_ = np.linalg.lstsq(A, dp, rcond=None)
    fit = A @ np.array([gamma, c0])
    assert abs(c0) < 0.05 * dp.min(), (c0, dp)  # through zero, up to the curvature correction of a diffuse interface
    assert np.abs(fit - dp).max() < 0.015 * dp.min(), (fit, dp)  # linear in 1/R
    ref = json.load(open(os.path.join(HERE, "golden", "sc_surface_tension.json")))["gamma"]
    assert gamma == pytest.approx(ref, rel=0.03)


@pytest.mark.slow
def test_low_zeta_electrophoretic_mobility_hueckel_hasimoto():
    L, r, Q, E = 20, 3.0, -2.0, 0.01
    p = synth.Params(nx=L, ny=L, nz=L, ncomp=1, nions=2, prec="fp64", tau=1.0, G=0.0, D=0.05, bjerrum=0.4,
                     eps_r=(1.0, 1.0), eps_r_colloid=1.0, E_ext=(E, 0.0, 0.0), poisson_tol=1e-10,
                     poisson_max_iter=200, ncolloid_max=1, colloids_move=0)
    cx = np.array([[L / 2 + 0.3, L / 2 - 0.2, L / 2 + 0.1]])
    kw = dict(colloid_x=cx, colloid_v=np.zeros((1, 3)), colloid_q=np.array([Q]), colloid_r=np.array([r]))
    rho = np.ones((1, L, L, L))
    fluid = OracleSystem(p, rho, np.zeros((2, L, L, L)), **kw).fluid
    n = np.zeros((2, L, L, L))
    n[0][fluid] = -Q / fluid.sum()  # counter-cations only, uniform over the fluid
    s = OracleSystem(p, rho, n, **kw)
    s.run(1300)
    mus = []
    phi = 4.0 / 3.0 * math.pi * r ** 3 / L ** 3
    for _ in range(3):
        s.run(100)
        mus.append(-(1.0 - phi) * float(s.last_u[0][s.fluid].mean()) / E)
    m1, m2, m3 = mus
    mu = (m1 * m3 - m2 * m2) / (m1 + m3 - 2.0 * m2)  # limit of the exponential approach
    eta = (1.0 / 3.0) * (s.tau - 0.5)
    kinv = (1.0 - 1.7601 * phi ** (1 / 3) + phi - 1.5593 * phi ** 2 + 3.9799 * phi ** (8 / 3)
            - 3.0734 * phi ** (10 / 3))
    mu_th = Q / (6.0 * math.pi * eta * r) * kinv
    assert mu < 0.0  # a negative sphere moves against the field
    assert mu == pytest.approx(mu_th, rel=0.15), (mu, mu_th, mus)

"""Physics validations of the oracle against the paper's Sec. III results.

Dielectric drop (Sec. III.B): an ion-free drop of the lower-permittivity
fluid in an applied field elongates along the field, and in the small
deformation limit delta = eps_a r chi^2 E^2 / (4 gamma) (O'Konski, eq.
droplet_deformation, quasi-2D geometry), with gamma from the Young-Laplace law
dp = gamma / r and the Shan-Chen equation of state p = c_s^2 rho +
c_s^2 G psi_a psi_b (eq. eqofstate).  The paper reports agreement within 15%
for small drops.  This pins the sign and size of the Kelvin force, the
polarisation of the permittivity by the applied field in the Poisson solve
and the Shan-Chen surface tension at once.
"""
import math

import numpy as np
import pytest

import synth
from oracle import OracleSystem
from oracle.model import psi_of


def _deformation_yz(rho, n):
    ra, rb = rho
    c = (rb - ra) / (ra + rb)
    w = np.maximum(c, 0.0).sum(axis=2)
    z, y = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    W = w.sum()
    yc, zc = (w * y).sum() / W, (w * z).sum() / W
    myy, mzz = (w * (y - yc) ** 2).sum(), (w * (z - zc) ** 2).sum()
    return (math.sqrt(mzz) - math.sqrt(myy)) / (math.sqrt(mzz) + math.sqrt(myy))


@pytest.mark.slow
def test_dielectric_drop_matches_okonski():
    n, r, G, E = 40, 10.0, 4.0, 0.2
    w = synth.droplet(n=n, r=r, G=G, Ez=0.0, nions=0, tol=1e-8, noise=0.0)
    w.params.nx = 2
    rho = w.rho[:, :, :, n // 2 - 1:n // 2 + 1].copy()
    s = OracleSystem(w.params, rho)
    s.run(600)
    ra, rb = s.densities()
    p = (ra + rb) / 3.0 + G / 3.0 * psi_of(ra) * psi_of(rb)
    c = n // 2
    dp = p[c, c, 0] - p[0, 0, 0]
    rd = math.sqrt(float(((rb - ra) > 0)[:, :, 0].sum()) / math.pi)
    gamma = dp * rd
    assert 0.03 < gamma < 0.2
    eps_a = 1.0 / (4.0 * math.pi * 0.4)
    chi = (1.0 - 0.5) / (1.0 + 0.5)
    delta_th = eps_a * rd * chi ** 2 * E ** 2 / (4.0 * gamma)
    s.E_ext = (0.0, 0.0, E)
    s.run(800)
    delta = _deformation_yz(s.densities(), n)
    assert delta > 0.0          # prolate along the field
    assert abs(delta / delta_th - 1.0) < 0.15

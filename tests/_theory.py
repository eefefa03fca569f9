"""Closed-form physics used by the physics checks (independent of the lattice
method and of both implementations).

Sharp-interface ion equilibrium at a flat fluid interface (Sec. III.A, after
Onuki): two semi-infinite electrolytes, fluid a for s < 0 and fluid b for
s > 0, permittivities eps_a, eps_b, Gibbs transfer energies dmu+ and dmu-.
In equilibrium n^(+-)(s) = n_a exp(-+ phi(s) - mu_s^(+-)(s)) with the
solvation potential 0 in fluid a and dmu^(+-) in fluid b (lattice units,
e = beta = 1, phi = 0 in bulk a).  Electroneutral bulks give
n_b = n_a exp(-(dmu+ + dmu-)/2) and the Donnan potential
phi_D = phi_b - phi_a = (dmu- - dmu+)/2.  In each fluid the Poisson equation
eps phi'' = -(n+ - n-) is the nonlinear Poisson-Boltzmann equation
psi'' = kappa^2 sinh(psi) about its bulk potential (kappa^2 = 2 n / eps, the
paper's screening length), whose decaying solution is the Gouy-Chapman
profile tanh(psi/4) = tanh(psi_0/4) exp(-kappa |s|).  The interface potential
phi_0 follows from continuity of eps phi' at s = 0:
eps_a kappa_a sinh(phi_0/2) = -eps_b kappa_b sinh((phi_0 - phi_D)/2).
(The paper quotes Bier's linearised form of this profile with an extra
interface shift; the nonlinear form needs no fitted parameter.)
"""
import math

import numpy as np


def sharp_interface(s, n_a, dmu, eps_a, eps_b):
    """phi(s), n+(s), n-(s) of the sharp-interface equilibrium; s is the signed
    distance from the interface (negative in fluid a), numpy array."""
    dp, dm = float(dmu[0]), float(dmu[1])
    n_b = n_a * math.exp(-0.5 * (dp + dm))
    phi_d = 0.5 * (dm - dp)
    ka = math.sqrt(2.0 * n_a / eps_a)
    kb = math.sqrt(2.0 * n_b / eps_b)

    def jump(p0):  # increasing in p0; its root is the interface potential
        return eps_a * ka * math.sinh(0.5 * p0) + eps_b * kb * math.sinh(0.5 * (p0 - phi_d))

    lo, hi = min(0.0, phi_d), max(0.0, phi_d)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if jump(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    p0 = 0.5 * (lo + hi)
    s = np.asarray(s, dtype=np.float64)
    in_a = s < 0.0
    psi_a = 4.0 * np.arctanh(math.tanh(0.25 * p0) * np.exp(-ka * np.abs(s)))
    psi_b = 4.0 * np.arctanh(math.tanh(0.25 * (p0 - phi_d)) * np.exp(-kb * np.abs(s)))
    phi = np.where(in_a, psi_a, phi_d + psi_b)
    mu_p = np.where(in_a, 0.0, dp)
    mu_m = np.where(in_a, 0.0, dm)
    n_p = n_a * np.exp(-phi - mu_p)
    n_m = n_a * np.exp(phi - mu_m)
    return phi, n_p, n_m


def flat_box_distance(nx):
    """Signed distance of cell x to the nearer interface of the periodic box
    with fluid a on x < nx/2 (interfaces at x = nx/2 - 1/2 and x = -1/2),
    negative in fluid a."""
    x = np.arange(nx, dtype=np.float64)
    h = nx // 2
    to_mid = x - (h - 0.5)
    to_edge = np.where(x < h, -(x + 0.5), (nx - 0.5) - x)
    return np.where(np.abs(to_mid) <= np.abs(to_edge), to_mid, to_edge)

"""Variable-permittivity Poisson equation (Sec. II.B eq. electric_potential,
Sec. II.D).  TEST INFRASTRUCTURE ONLY.

Discrete equation for the internal potential phi_I (symmetric seven-point
flux form, periodic), written for the total potential phi_I - E_ext.x so that
the applied field polarises the variable permittivity:

    sum_{d in Q6} eps_{i+d/2} (phi_{i+d} - phi_i)
        = -(q_i - qbar) + sum_{d in Q6} eps_{i+d/2} (E_ext . c_d),
    eps_{i+d/2} = (eps_i + eps_{i+d}) / 2,   mean(phi) = 0.

Reading: eq. electric_potential prints only phi_I; with the external part left
out an ion-free dielectric drop (Sec. III.B) would see a uniform field and
could not deform, while the paper reports its deformation and the bending of
the field lines around it.  The last term is the discrete divergence of
eps E_ext and has zero mean.

Solver: the paper's split of Sec. II.D -- a constant-coefficient Poisson
problem inverted spectrally, with the variable-permittivity part moved to the
right-hand side and taken from the previous iterate -- iterated to convergence
instead of lagged one step:

    eps0 L phi^{k+1} = -(q - qbar) - div_h((eps - eps0) grad_h phi^k),
    eps0 = (eps_max + eps_min) / 2,

with L the seven-point Laplacian inverted by FFT through its exact symbol
-sum_a 2(1 - cos(2 pi k_a / n_a)) (k = 0 mode set to zero).  Reading: the
paper's printed split drops the 1/eps on the grad(eps).grad(phi) term; the
flux form above is the consistent discrete statement, and at convergence the
iteration gives its unique mean-zero solution.  Stop rule:
||b - A phi||_2 / ||b||_2 < tol.
"""
import numpy as np

from .lattice import AXES, shift


def flux_operator(phi, eps):
    """(A_eps phi)_i = sum_a [eps_{i+a/2}(phi_{i+a}-phi_i) - eps_{i-a/2}(phi_i-phi_{i-a})]."""
    out = np.zeros_like(phi)
    for a in range(3):
        e = AXES[a]
        ef = 0.5 * (eps + shift(eps, e))
        flux = ef * (shift(phi, e) - phi)
        out += flux - shift(flux, -e)
    return out


def laplacian_symbol(shape):
    """Eigenvalues of the periodic seven-point Laplacian, indexed like fftn."""
    nz, ny, nx = shape
    kz = 2.0 * (1.0 - np.cos(2.0 * np.pi * np.arange(nz) / nz))
    ky = 2.0 * (1.0 - np.cos(2.0 * np.pi * np.arange(ny) / ny))
    kx = 2.0 * (1.0 - np.cos(2.0 * np.pi * np.arange(nx) / nx))
    return -(kz[:, None, None] + ky[None, :, None] + kx[None, None, :])


def solve_laplace(g):
    """Mean-zero phi with L phi = g (g must have zero mean)."""
    lam = laplacian_symbol(g.shape)
    gh = np.fft.fftn(g)
    lam0 = lam.copy()
    lam0[0, 0, 0] = 1.0
    ph = gh / lam0
    ph[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(ph))


def external_source(eps, E_ext):
    """sum_{d in Q6} eps_{i+d/2} (E_ext . c_d) = sum_a E_a (eps_{i+a/2} - eps_{i-a/2})."""
    out = np.zeros_like(eps)
    for a in range(3):
        if E_ext[a] != 0.0:
            e = AXES[a]
            ef = 0.5 * (eps + shift(eps, e))
            out += E_ext[a] * (ef - shift(ef, -e))
    return out


def solve(q, eps, phi0=None, tol=1e-10, max_iter=500, E_ext=(0.0, 0.0, 0.0)):
    """Solve the flux-form Poisson equation.  Returns (phi, iterations, relres).

    If the right-hand side vanishes, phi = 0 and zero iterations are taken."""
    b = -(q - q.mean()) + external_source(eps, E_ext)
    bn = float(np.sqrt((b * b).sum()))
    if bn == 0.0:
        return np.zeros_like(q), 0, 0.0
    eps0 = 0.5 * (float(eps.max()) + float(eps.min()))
    phi = np.zeros_like(q) if phi0 is None else phi0 - phi0.mean()
    r = b - flux_operator(phi, eps)
    relres = float(np.sqrt((r * r).sum())) / bn
    it = 0
    while relres >= tol and it < max_iter:
        g = (b - flux_operator(phi, eps - eps0)) / eps0
        g -= g.mean()
        phi = solve_laplace(g)
        r = b - flux_operator(phi, eps)
        relres = float(np.sqrt((r * r).sum())) / bn
        it += 1
    return phi, it, relres

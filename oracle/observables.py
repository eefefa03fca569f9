"""Observables of a lattice system.  TEST INFRASTRUCTURE ONLY.

* component masses, ion totals, net charge and fluid momentum (conservation
  checks of Sec. II: the flux-form ion update and the bounce-back conserve
  ions, charge and fluid mass exactly);
* droplet deformation D = (sqrt(M_zz) - sqrt(M_xx)) / (sqrt(M_zz) + sqrt(M_xx))
  from second moments of the weight w = max(0, c), c = (rho_b - rho_a) /
  (rho_a + rho_b), about the weighted centroid (the drop must not cross the
  periodic boundary).  The paper's deformation delta = (b - a)/(b + a)
  (Sec. III.B) is the same ratio for an ellipse when the semi-axes are taken
  proportional to the square roots of the second moments.
"""
import numpy as np

from .lattice import C, Q


def conserved(sys):
    fl = sys.fluid
    rho = sys.f.sum(axis=1) * fl
    mass = [float(rho[s].sum()) for s in range(sys.ncomp)]
    ions = [float(sys.n[s].sum()) for s in range(sys.n.shape[0])]
    charge = float(sys.qc.sum())
    if sys.nions:
        charge += ions[0] - ions[1]
    mom = np.zeros(3)
    for q in range(1, Q):
        s = float((sys.f[:, q] * fl).sum())
        mom += C[q] * s
    return {"mass": mass, "ions": ions, "charge": charge, "momentum": mom.tolist()}


def deformation(rho):
    """rho: (2, nz, ny, nx).  Returns (D, centroid (x, y, z))."""
    ra, rb = rho[0], rho[1]
    tot = ra + rb
    c = np.where(tot > 0, (rb - ra) / np.where(tot > 0, tot, 1.0), 0.0)
    w = np.maximum(c, 0.0)
    nz, ny, nx = ra.shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    W = w.sum()
    if W == 0:
        return 0.0, (0.0, 0.0, 0.0)
    xc, yc, zc = (w * x).sum() / W, (w * y).sum() / W, (w * z).sum() / W
    mxx = (w * (x - xc) ** 2).sum()
    mzz = (w * (z - zc) ** 2).sum()
    a, b = np.sqrt(mxx), np.sqrt(mzz)
    return float((b - a) / (b + a)), (float(xc), float(yc), float(zc))

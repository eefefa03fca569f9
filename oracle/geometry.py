"""Projection of spherical colloids onto the lattice (Sec. II.E).
TEST INFRASTRUCTURE ONLY.

* A node is solid when its centre lies strictly inside a sphere (minimum-image
  distance squared < r^2, evaluated in FP64 without fused multiply-add, ties
  go to fluid) -- "marking as solid the sites that are covered by the
  particle" (Sec. II.E, projection paragraph).
* Solid fraction psi_s = nu/(h+1)^3 with nu the number of sub-cube centres
  (h+1 per axis) strictly inside the sphere (Sec. II.E, partial-volume
  paragraph).  The paper does not give h; reading: h = 3 (64 samples).
* Surface nodes: solid nodes with at least one fluid D3Q19 neighbour; these
  also are the interface nodes that carry the virtual fluid density
  (Sec. II.E, Jansen correction).
* Colloid charge: Q split equally over the colloid's surface nodes (the
  workloads place the charge on surface nodes instead of the volume
  distribution Q psi_s / v_p of Sec. II.E).
"""
import numpy as np

from .lattice import C, Q, shift


def min_image(d, n):
    """Minimum-image wrap of a coordinate difference (exact in FP64)."""
    d = np.where(d > 0.5 * n, d - n, d)
    d = np.where(d < -0.5 * n, d + n, d)
    return d


def _dist2(px, py, pz, X, nx, ny, nz):
    dx = min_image(px - X[0], nx)
    dy = min_image(py - X[1], ny)
    dz = min_image(pz - X[2], nz)
    # ((dx*dx + dy*dy) + dz*dz), each product and sum rounded separately
    return (dx * dx + dy * dy) + dz * dz


def project(nx, ny, nz, X, R, h=3):
    """Solid mask, owner id (-1 for fluid) and solid fraction psi_s.

    X: (N, 3) centres (x, y, z); R: (N,) radii."""
    shape = (nz, ny, nx)
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    solid = np.zeros(shape, dtype=bool)
    owner = np.full(shape, -1, dtype=np.int64)
    psi_s = np.zeros(shape)
    offs = [(k + 0.5) / (h + 1) - 0.5 for k in range(h + 1)]
    for j in range(len(R)):
        r2 = R[j] * R[j]
        inside = _dist2(x, y, z, X[j], nx, ny, nz) < r2
        solid |= inside
        owner[inside] = j
        nu = np.zeros(shape)
        for oz in offs:
            for oy in offs:
                for ox in offs:
                    nu += _dist2(x + ox, y + oy, z + oz, X[j], nx, ny, nz) < r2
        psi_s += nu / float((h + 1) ** 3)
    psi_s = np.minimum(psi_s, 1.0)
    return solid, owner, psi_s


def project_boxed(nx, ny, nz, X, R, h=3):
    """The projection of `project`, evaluated only on each sphere's bounding
    box (every node or sub-cube centre farther than r + 1 from the centre
    along an axis lies outside the sphere), so that large boxes with many
    spheres stay affordable.  Same per-node arithmetic and the same owner rule
    (the last sphere containing a node owns it)."""
    shape = (nz, ny, nx)
    dims = (nx, ny, nz)
    solid = np.zeros(shape, dtype=bool)
    owner = np.full(shape, -1, dtype=np.int64)
    psi_s = np.zeros(shape)
    offs = [(k + 0.5) / (h + 1) - 0.5 for k in range(h + 1)]
    for j in range(len(R)):
        r2 = R[j] * R[j]
        axes = []
        for a in range(3):
            lo = int(np.ceil(X[j][a] - R[j] - 1.0))
            hi = int(np.floor(X[j][a] + R[j] + 1.0))
            idx = np.arange(lo, hi + 1) % dims[a]
            axes.append(np.unique(idx))
        ix, iy, iz = axes
        z, y, x = np.meshgrid(iz.astype(np.float64), iy.astype(np.float64), ix.astype(np.float64), indexing="ij")
        sel = np.ix_(iz, iy, ix)
        inside = _dist2(x, y, z, X[j], nx, ny, nz) < r2
        s = solid[sel]
        o = owner[sel]
        s |= inside
        o[inside] = j
        solid[sel] = s
        owner[sel] = o
        nu = np.zeros(inside.shape)
        for oz in offs:
            for oy in offs:
                for ox in offs:
                    nu += _dist2(x + ox, y + oy, z + oz, X[j], nx, ny, nz) < r2
        psi_s[sel] += nu / float((h + 1) ** 3)
    psi_s = np.minimum(psi_s, 1.0)
    return solid, owner, psi_s


def surface_nodes(solid):
    """Solid nodes with at least one fluid D3Q19 neighbour."""
    fluid = ~solid
    has_fluid_nb = np.zeros_like(solid)
    for q in range(1, Q):
        has_fluid_nb |= shift(fluid, C[q])
    return solid & has_fluid_nb


def colloid_charge(owner, surface, charges):
    """q_c: colloid charge Q_j spread equally over its surface nodes."""
    qc = np.zeros(owner.shape)
    for j, Qj in enumerate(charges):
        m = surface & (owner == j)
        cnt = int(m.sum())
        if cnt > 0:
            qc[m] = Qj / cnt
    return qc


def boundary_links(solid, owner):
    """Sorted list of (node index, q, colloid id) for every fluid node whose
    D3Q19 neighbour x + c_q is solid (the halfway bounce-back links)."""
    fluid = ~solid
    out = []
    for q in range(1, Q):
        nb_solid = shift(solid, C[q])
        nb_owner = shift(owner, C[q])
        idx = np.flatnonzero((fluid & nb_solid).ravel())
        for i in idx:
            out.append((int(i), q, int(nb_owner.ravel()[i])))
    out.sort()
    return out

"""Pins of the oracle's colloid dynamics (Sec. II.E) and of the drop
deformation observable (Sec. III.B) against results that do not come from the
oracle itself.

* Hertz contact (eq. colloid_interaction): the pair force is minus the
  gradient of the Hertz contact energy V(delta) = (2/5) k_H delta^{5/2},
  differentiated numerically with respect to one centre, so a wrong exponent,
  prefactor or sign of the force fails; equal and opposite along the line of
  centres; zero without overlap.
* Lubrication (eq. lubrication): Reynolds' lubrication law for two equal
  spheres of radius a approaching at normal speed v across a gap h -> 0,
  |F| h -> (3/2) pi eta a^2 |v| (lubrication theory, not the paper's text);
  the force opposes the normal relative motion, ignores tangential motion,
  is antisymmetric and acts only inside the gap window 0 < h < 2/3.
* Velocity-Verlet (Sec. II.E, Newton's equation): a colloid under a constant
  force F moves as x0 + v0 t + F t^2 / (2m) and v0 + F t / m exactly, with
  m = rho_p (4/3) pi r^3, through the oracle's move-and-remap routine.
* Deformation: for a uniform ellipsoid with semi-axes (a, a, b) the second
  moments give sqrt(M_zz / M_xx) = b / a (moments of a solid ellipsoid), so the
  observable tends to (b - a)/(b + a) as the lattice resolves the ellipsoid;
  a sphere gives zero, an ellipsoid along x a negative value.
"""
import math

import numpy as np
import pytest

import synth
from oracle import colloids, observables
from oracle.model import OracleSystem


# ---------------------------------------------------------------- Hertz
def _hertz_energy(xi, xj, r, k, dims):
    d = np.array([colloids.min_image(xi[a] - xj[a], dims[a]) for a in range(3)])
    delta = max(2.0 * r - float(np.sqrt((d * d).sum())), 0.0)
    return 0.4 * k * delta ** 2.5


@pytest.mark.parametrize("overlap", [0.05, 0.3, 0.9])
def test_hertz_force_is_minus_gradient_of_contact_energy(overlap):
    r, k, dims = 3.0, 1.7, (20, 20, 20)
    rng = np.random.default_rng(11)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    xj = np.array([10.0, 10.0, 10.0])
    xi = xj + (2.0 * r - overlap) * n
    X = np.stack([xi, xj])
    F = colloids.pair_forces(X, np.zeros((2, 3)), np.array([r, r]), dims, k, eta=0.0)
    h = 1e-6
    grad = np.zeros(3)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        grad[a] = (_hertz_energy(xi + e, xj, r, k, dims) - _hertz_energy(xi - e, xj, r, k, dims)) / (2 * h)
    assert np.allclose(F[0], -grad, rtol=1e-6, atol=1e-12), (F[0], -grad)
    assert np.allclose(F[1], -F[0], rtol=0, atol=1e-15)
    # along the line of centres, pushing i away from j
    assert float(F[0] @ n) > 0 and np.linalg.norm(np.cross(F[0], n)) < 1e-12 * np.linalg.norm(F[0])


def test_hertz_force_vanishes_without_overlap_and_wraps_periodically():
    r, k, dims = 3.0, 1.0, (16, 16, 16)
    X = np.array([[1.0, 8.0, 8.0], [15.0 - 0.5, 8.0, 8.0]])  # 2.5 apart across the x boundary
    F = colloids.pair_forces(X, np.zeros((2, 3)), np.array([r, r]), dims, k, eta=0.0)
    delta = 2 * r - 2.5
    assert F[0][0] == pytest.approx(k * delta ** 1.5, rel=1e-12)  # i is at larger x in the minimum image
    X = np.array([[2.0, 8.0, 8.0], [8.5, 8.0, 8.0]])  # 6.5 apart: no contact
    F = colloids.pair_forces(X, np.zeros((2, 3)), np.array([r, r]), dims, k, eta=0.0)
    assert np.all(F == 0.0)


# ---------------------------------------------------------------- lubrication
def _lub(gap, vi, vj, r=4.0, eta=1.0 / 6.0, dims=(64, 64, 64), k=0.0):
    xj = np.array([20.0, 30.0, 30.0])
    xi = xj + np.array([2.0 * r + gap, 0.0, 0.0])
    return colloids.pair_forces(np.stack([xi, xj]), np.stack([vi, vj]), np.array([r, r]), dims, k, eta)


def test_lubrication_reynolds_limit_for_equal_spheres():
    r, eta, v = 4.0, 1.0 / 6.0, 1e-3
    reynolds = 1.5 * math.pi * eta * r * r * v  # |F| h as h -> 0
    for gap in (1e-3, 1e-4, 1e-5):
        F = _lub(gap, np.array([-v, 0, 0]), np.zeros(3), r, eta)
        assert abs(F[0][0]) * gap == pytest.approx(reynolds, rel=2 * gap)


def test_lubrication_opposes_normal_motion_only_inside_its_window():
    v = np.array([-2e-3, 0.0, 0.0])  # i approaches j along -x
    for gap in (0.05, 0.2, 0.5, 0.6):
        F = _lub(gap, v, np.zeros(3))
        assert F[0][0] > 0.0  # repels the approaching sphere
        assert float(F[0] @ v) < 0.0  # dissipative
        assert np.allclose(F[1], -F[0], rtol=0, atol=1e-18)
        Fs = _lub(gap, -v, np.zeros(3))  # separating: pulled back
        assert Fs[0][0] < 0.0 and Fs[0][0] == pytest.approx(-F[0][0], rel=1e-14)
        Ft = _lub(gap, np.array([0.0, 3e-3, -1e-3]), np.zeros(3))  # tangential motion
        assert np.all(np.abs(Ft) < 1e-18)
    for gap in (0.667, 0.8, 1.5):
        assert np.all(_lub(gap, v, np.zeros(3)) == 0.0)
    # the bracket (1/h - 1) of eq. lubrication vanishes at h = 1 and is 1 at h = 1/2
    F = _lub(0.5, v, np.zeros(3), r=4.0, eta=1.0 / 6.0)
    assert F[0][0] == pytest.approx(1.5 * math.pi / 6.0 * 16.0 * 2e-3, rel=1e-12)


# ---------------------------------------------------------------- Verlet
def test_velocity_verlet_under_constant_force_follows_the_closed_form():
    n, r, rho_p = 16, 3.0, 5.0
    p = synth.Params(nx=n, ny=n, nz=n, ncomp=1, nions=0, prec="fp64", G=0.0, ncolloid_max=1,
                     colloids_move=1, rho_p=rho_p)
    x0 = np.array([[5.25, 7.5, 8.125]])
    v0 = np.array([[0.03, -0.01, 0.02]])
    # empty lattice (zero density): no fluid momentum to exchange in the remap
    s = OracleSystem(p, np.zeros((1, n, n, n)), colloid_x=x0, colloid_v=v0, colloid_q=np.zeros(1),
                     colloid_r=np.array([r]))
    m = rho_p * 4.0 / 3.0 * math.pi * r ** 3
    F = np.array([[2.0, -1.0, 0.5]])
    for t in range(1, 41):
        s.colloid_force = F.copy()
        colloids.move_and_remap(s)
        x = (x0 + v0 * t + F * t * t / (2.0 * m)) % n
        assert np.allclose(s.cx, x, rtol=0, atol=1e-12), (t, s.cx, x)
        assert np.allclose(s.cv, v0 + F * t / m, rtol=0, atol=1e-15)
    assert s.cmass[0] == pytest.approx(m, rel=1e-15)


# ---------------------------------------------------------------- contact
def _pair_at_rest(dist, r=5.0):
    nx, ny, nz = 36, 24, 24
    p = synth.Params(nx=nx, ny=ny, nz=nz, ncomp=1, nions=0, prec="fp64", G=0.0, ncolloid_max=2, colloids_move=0)
    cx = np.array([[nx / 2 - dist / 2, 12.3, 12.1], [nx / 2 + dist / 2, 12.3, 12.1]])
    s = OracleSystem(p, np.ones((1, nz, ny, nx)), colloid_x=cx, colloid_v=np.zeros((2, 3)),
                     colloid_q=np.zeros(2), colloid_r=np.full(2, r))
    s.step()
    return s.colloid_force


def test_touching_spheres_are_pushed_together_beyond_the_hertz_force():
    """Two fixed spheres (r = 5) in fluid at rest: while fluid nodes separate
    them the boundary-link forces cancel; once no fluid node is left between
    them, the outer fluid's pressure pushes each toward the other, and at the
    stiffness k_H = 1 that Sec. II.E takes this exceeds the Hertz repulsion
    k_H delta^{3/2} several times over (so two spheres pressed into contact
    keep closing instead of resting at a small overlap)."""
    for dist in (10.6, 10.0):
        F = _pair_at_rest(dist)
        assert np.abs(F).max() < 1e-10, (dist, F)
    for dist in (9.6, 9.2):
        F = _pair_at_rest(dist)
        delta = 10.0 - dist
        assert np.allclose(F[0], -F[1], rtol=0, atol=1e-12)  # equal and opposite
        assert abs(F[0, 1]) < 1e-10 and abs(F[0, 2]) < 1e-10  # along the line of centres
        hertz = 1.0 * delta ** 1.5
        # net force (pressure part minus the Hertz repulsion) toward the other
        # sphere by more than twice the repulsion: the pressure part is over
        # three times the Hertz force (measured: 9.3x at overlap 0.4, 5.6x at 0.8)
        assert F[0, 0] > 2.0 * hertz, (dist, F[0, 0], hertz)


# ---------------------------------------------------------------- deformation
def _ellipsoid_rho(n, ax, ay, az, centre):
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    inside = ((x - centre[0]) / ax) ** 2 + ((y - centre[1]) / ay) ** 2 + ((z - centre[2]) / az) ** 2 < 1.0
    return np.stack([np.where(inside, 0.0, 1.0), np.where(inside, 1.0, 0.0)])  # c = +1 inside, -1 outside


@pytest.mark.parametrize("a,b", [(10.0, 14.0), (12.0, 9.0), (11.0, 11.0)])
def test_deformation_of_a_sharp_ellipsoid(a, b):
    n = 48
    c = (23.7, 24.2, 23.9)  # off-lattice centre: no symmetric cancellation of the sampling error
    D, cen = observables.deformation(_ellipsoid_rho(n, a, a, b, c))
    exact = (b - a) / (b + a)
    assert D == pytest.approx(exact, abs=4e-3), (D, exact)
    assert np.allclose(cen, c, atol=2e-2)


def test_deformation_sign_and_weight():
    n = 40
    c = (19.5, 20.0, 20.5)
    D_x, _ = observables.deformation(_ellipsoid_rho(n, 12.0, 9.0, 9.0, c))  # long along x
    assert D_x == pytest.approx((9.0 - 12.0) / (9.0 + 12.0), abs=5e-3)
    rho = _ellipsoid_rho(n, 9.0, 9.0, 12.0, c)
    D0, _ = observables.deformation(rho)
    # the weight is max(0, c): scaling the outside (c < 0) region changes nothing
    rho2 = rho.copy()
    rho2[0] *= 3.0
    D2, _ = observables.deformation(rho2)
    assert D2 == D0
    # half-weight interface cells (c = 0.5 -> w = 0.5) enter the moments linearly
    rho3 = rho.copy()
    rho3[0][rho[1] > 0] = 1.0 / 3.0  # inside: c = (1 - 1/3)/(1 + 1/3) = 0.5, uniform weight 0.5
    D3, _ = observables.deformation(rho3)
    assert D3 == pytest.approx(D0, abs=1e-13)

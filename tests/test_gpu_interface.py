"""A sphere at a fluid interface (Sec. III.F): a neutral sphere of radius 8
in a 64^3 box with two flat Shan-Chen interfaces, moving with velocity-Verlet
and bounce-back coupling to both fluids, the interface solid nodes carrying
the mean density of their fluid neighbours (neutral wetting, contact angle
90 degrees).

* Interface: a sphere started at the interface stays there (|dz| < 1e-3
  over 6000 steps); one started 3 cells into fluid b is pulled back through
  the interface within 500 steps (measured: from +3 to -1.3 cells).
* Salt (Gibbs transfer energies +4 kT for both species, so the ions stay in
  fluid a; salt 1e-3 and 2e-3): the sphere leaves its salt-free position
  toward fluid a, and its displacement after 1000 steps is proportional to
  the salt concentration (measured 0.60 and 1.22 cells), the paper's
  observation of a displacement linear in the salt.  Unlike the paper's
  runs, the sphere does not settle at a displaced equilibrium here: it keeps
  moving into fluid a over 8000 steps (measured 15.5 cells at 1e-3).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _track(lbeh, w, steps, every):
    s = lbeh.System(w.params)
    s.set_fields(rho=list(w.rho), n=list(w.n) if w.n is not None else None, colloid_x=w.colloid_x,
                 colloid_v=w.colloid_v, colloid_q=w.colloid_q, colloid_r=w.colloid_r)
    z = []
    for _ in range(steps // every):
        assert s.step(every) == lbeh.LBEH_OK
        z.append(float(np.array(s.get(("rho",))["cx"])[0, 2]))
    o = s.observables()
    s.close()
    return np.array(z), o


def test_sphere_at_the_interface(lbeh):
    n = 64
    zi = n / 2.0 - 0.5
    z_off, _ = _track(lbeh, synth.interface_colloid(n=n, dz=3.0), 2000, 500)
    z_on, _ = _track(lbeh, synth.interface_colloid(n=n, dz=0.0), 6000, 500)
    print("interface", z_off - zi, z_on - zi)
    assert z_off[0] - zi < 0.0  # pulled back through the interface from +3
    assert np.abs(z_on - zi).max() < 1e-3  # a sphere at the interface stays there


def test_salt_displaces_the_sphere_in_proportion(lbeh):
    n = 64
    zi = n / 2.0 - 0.5
    d = []
    for salt in (1e-3, 2e-3):
        z, o = _track(lbeh, synth.interface_colloid(n=n, dz=0.0, salt=salt), 1000, 1000)
        assert o.status == lbeh.LBEH_OK
        d.append(float(z[-1] - zi))
    print("salt displacements", d)
    assert d[0] < -0.2 and d[1] < -0.2  # toward fluid a
    assert 1.7 < d[1] / d[0] < 2.3, d  # linear in the salt concentration


def test_colloid_coated_droplet(lbeh):
    """Sec. III.G: 80 uncharged spheres (radius 5) adsorbed on a drop of
    radius 32 (covering fraction 0.49) in the charged-drop setting of
    Sec. III.D (salt 1e-3, transfer energies +-4 kT, E_z = 1e-3), 128^3,
    FP32, 3000 steps: every sphere still straddles the interface (its centre
    closer than r_p to the drop's equimolar radius around the drop centroid;
    measured at most 2.2-2.4 cells every 500 steps, the equimolar radius of
    fluid b being 30.2 with the spheres taking part of the drop's volume), no
    two spheres interpenetrate by more than Hertz contact allows (measured
    closest centres 10.004: the coating is packed), the ions are conserved
    (measured 2.5e-9) and the solve converges at every step."""
    w = synth.coated_droplet(n=128)
    s = lbeh.System(w.params)
    s.set_fields(rho=list(w.rho), n=list(w.n), colloid_x=w.colloid_x, colloid_v=w.colloid_v,
                 colloid_q=w.colloid_q, colloid_r=w.colloid_r)
    o0 = s.observables()
    worst = []
    for _ in range(6):
        assert s.step(500) == lbeh.LBEH_OK
        g = s.get(("rho",))
        cx = np.array(g["cx"])
        o = s.observables()
        ra, rb = g["rho"]
        vol = float(((rb - ra) > 0).sum())  # fluid b: the drop
        req = (3.0 * vol / (4.0 * np.pi)) ** (1.0 / 3.0)
        d = cx - np.asarray(o.centroid)
        d -= 128.0 * np.round(d / 128.0)
        rad = np.sqrt((d * d).sum(axis=1))
        pair = np.sqrt(((cx[:, None, :] - cx[None, :, :]) ** 2).sum(-1))
        np.fill_diagonal(pair, np.inf)
        worst.append((float(np.abs(rad - req).max()), float(pair.min()), req))
    o1 = s.observables()
    s.close()
    print("coated droplet", worst)
    mass = max(abs(o1.mass[k] / o0.mass[k] - 1.0) for k in range(2))
    ions = max(abs(o1.ions[k] / o0.ions[k] - 1.0) for k in range(2))
    print("conservation", mass, ions)
    # ions are remapped exactly when the spheres cover and uncover nodes; the
    # fluid mass of covered nodes is not (new fluid nodes take their
    # neighbours' density): measured 1.4e-4 over 3000 steps
    assert ions < 1e-6 and mass < 1e-3
    for dev, dmin, _ in worst:
        assert dev < 5.0, worst  # r_p: the sphere still crosses the interface
        assert dmin > 2 * 5.0 - 0.5, worst

"""A sphere at a fluid interface (Sec. III.F): a neutral sphere of radius 8
in a 64^3 box with two flat Shan-Chen interfaces, moving with velocity-Verlet
and bounce-back coupling to both fluids, the interface solid nodes carrying
the mean density of their fluid neighbours (neutral wetting, contact angle
90 degrees).

* Trapping: a sphere started 3 cells into fluid b is pulled back toward the
  interface (capillary restoring force) and one started at the interface
  stays there.
* Salt (Gibbs transfer energies +4 kT for both species, so the ions stay in
  fluid a): the ions' osmotic pressure displaces the sphere from its salt-free
  position, more at the higher concentration (the paper reports a
  displacement linear in the salt concentration).
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


def test_sphere_is_trapped_at_the_interface(lbeh):
    n = 64
    zi = n / 2.0 - 0.5
    z_off, _ = _track(lbeh, synth.interface_colloid(n=n, dz=3.0), 6000, 500)
    z_on, _ = _track(lbeh, synth.interface_colloid(n=n, dz=0.0), 6000, 500)
    print("trap", z_off - zi, z_on - zi)
    assert abs(z_off[-1] - zi) < 2.0  # pulled back from 3 cells into fluid b
    assert np.all(np.diff(np.abs(z_off - zi))[:4] < 0.0)  # moving toward the interface
    assert np.abs(z_on - zi).max() < 0.5  # stays at the interface


def test_salt_displaces_the_sphere(lbeh):
    n = 64
    zs = []
    for salt in (0.0, 1e-3, 2e-3):
        z, o = _track(lbeh, synth.interface_colloid(n=n, dz=0.0, salt=salt), 8000, 1000)
        zs.append(float(z[-3:].mean()))
        print("salt", salt, z - (n / 2.0 - 0.5), o.status)
    d1, d2 = abs(zs[1] - zs[0]), abs(zs[2] - zs[0])
    print("displacements", d1, d2)
    assert d2 > d1 > 0.05

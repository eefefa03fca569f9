"""The paper's own validation settings on the GPU (Sec. III.A, III.B).

* Flat interfaces with selective solvation (Sec. III.A): the paper's
  quasi-one-dimensional box (512 x 4 x 4 here: the paper's 500 is not a
  length the transforms or the multigrid halve to small coarse levels), salt
  1e-3 in fluid a and the Donnan-balanced 1e-3 exp(-(dmu+ + dmu-)/2) in fluid
  b, Gibbs transfer energies dmu+- = +-dmu for dmu in {1, 3, 5} kT and
  permittivity contrasts chi in {0, 0.5, 0.9}: after the double layers have
  formed, the bulk potential difference is the Donnan potential and the ion
  profiles follow the sharp-interface (Gouy-Chapman) equilibrium of
  tests/_theory.py.  The paper reports < 5% deviation from its linearised
  profile over this range; the measured deviations and the bounds asserted
  are stated below.
* Dielectric drops in the paper's quasi-2D geometry at its other box size
  and radii (Sec. III.B: l in {64, 128}, r/l in {0.1, 0.25}): the
  stationary deformation against delta = eps_a r chi^2 E^2 / (4 gamma)
  (eq. droplet_deformation); the paper reports excellent agreement for r >= 30
  and up to 15% deviation for small drops.
"""
import copy
import json
import math
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _flat(lbeh, dmu, chi, steps, prec="fp64"):
    from _theory import flat_box_distance, sharp_interface
    coex = json.load(open(os.path.join(GOLD, "sc_coexistence.json")))
    nx, salt = 512, 1e-3
    drho0 = coex["rho_major"] - coex["rho_minor"]
    w = synth.flat_interface(nx=nx, ny=4, nz=4, dmu=(dmu, -dmu), chi=chi, salt=salt, drho_a=drho0, tol=1e-7,
                             rho_major=coex["rho_major"], rho_minor=coex["rho_minor"], prec=prec)
    s = lbeh.System(w.params)
    s.set_fields(rho=list(w.rho), n=list(w.n))
    assert s.step(steps) == lbeh.LBEH_OK
    out = s.get(("rho", "n", "phi"))
    o = s.observables()
    s.close()
    n, phi, ra = out["n"][:, 0, 0], out["phi"][0, 0], out["rho"][0, 0, 0]
    ratio = float(ra[nx // 4] - ra[3 * nx // 4]) / drho0
    de = (dmu * ratio, -dmu * ratio)
    eps_a = 1.0 / (4.0 * math.pi * 0.4)
    eps_b = eps_a * (1.0 - chi) / (1.0 + chi)
    sd = flat_box_distance(nx)
    total = float(n.sum())
    lo, hi = 0.5 * salt, 2.0 * salt
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        _, p_, m_ = sharp_interface(sd, mid, de, eps_a, eps_b)
        lo, hi = (lo, mid) if float((p_ + m_).sum()) > total else (mid, hi)
    _, n_p, n_m = sharp_interface(sd, 0.5 * (lo + hi), de, eps_a, eps_b)
    far = np.abs(sd) > 5.0
    err = max(float((np.abs(n[0] - n_p) / n_p)[far].max()), float((np.abs(n[1] - n_m) / n_m)[far].max()))
    donnan = float(phi[3 * nx // 4] - phi[nx // 4])
    mom = float(np.abs(np.asarray(o.momentum)).max())
    return {"donnan_rel": donnan / (0.5 * (de[1] - de[0])) - 1.0, "profile": err, "momentum": mom}


# Measured in FP64 after 15 000 steps (slabs at rest; relative deviations
# from the sharp-interface equilibrium, Donnan potential / ion profiles more
# than 5 cells from the interfaces):
#   dmu = 1: chi 0, 0.5, 0.9 -> 0.4%, 0.5%, 0.5% / 2.3%, 3.0%, 9.1%
#   dmu = 3: chi 0, 0.5, 0.9 -> 2.4%, 3.7%, 4.0% / 11%, 25%, 100%
#   dmu = 5: chi 0, 0.5, 0.9 -> 2.1%, 5.6%, 7.7% / 38%, 116%, 630%
# The Donnan potential stays within 8% over the paper's range.  The ion
# profiles near the interfaces reproduce the paper's "< 5%" only at dmu = 1
# (chi <= 0.5): at larger transfer energies the link-flux equilibrium across
# the ~4-cell Shan-Chen interface, whose per-link zero-flux ratio
# (1 - w/2)/(1 + w/2) approximates exp(-w) only for small w ~ dmu/4, departs
# from the sharp-interface profile that has no fitted parameter (the paper
# compares with a linearised profile and a fitted interface shift).  Bounds:
# the Donnan potential everywhere, the profiles at dmu = 1.  Beyond ~2e4 steps
# a uniform-flow mode of the coupled discrete equations grows from round-off
# (faster with permittivity contrast) and translates the slabs; the momentum
# bound asserts that the comparison is taken before it.
DONNAN_BOUND = {1.0: 0.01, 3.0: 0.05, 5.0: 0.10}
PROFILE_BOUND = {(1.0, 0.0): 0.04, (1.0, 0.5): 0.05, (1.0, 0.9): 0.12}


@pytest.mark.parametrize("dmu", [1.0, 3.0, 5.0])
@pytest.mark.parametrize("chi", [0.0, 0.5, 0.9])
def test_flat_interface_paper_sweep(lbeh, dmu, chi):
    r = _flat(lbeh, dmu, chi, 15000)
    print("flat512 dmu=%g chi=%g" % (dmu, chi), r)
    assert r["momentum"] < 1e-3, r  # slabs at rest: the profiles are comparable
    assert abs(r["donnan_rel"]) < DONNAN_BOUND[dmu], r
    if (dmu, chi) in PROFILE_BOUND:
        assert r["profile"] < PROFILE_BOUND[(dmu, chi)], r


def _deformation_yz(rho, n):
    ra, rb = rho
    c = (rb - ra) / (ra + rb)
    w = np.maximum(c, 0.0).sum(axis=2)
    z, y = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    W = w.sum()
    yc, zc = (w * y).sum() / W, (w * z).sum() / W
    myy, mzz = (w * (y - yc) ** 2).sum(), (w * (z - zc) ** 2).sum()
    return (math.sqrt(mzz) - math.sqrt(myy)) / (math.sqrt(mzz) + math.sqrt(myy))


@pytest.mark.parametrize("n,rl", [(64, 0.25), (64, 0.1), (128, 0.1)])
def test_quasi_2d_drop_other_sizes(lbeh, n, rl):
    gamma = json.load(open(os.path.join(GOLD, "sc_surface_tension.json")))["gamma"]
    eps_b, E = 0.5, 0.08
    r = rl * n
    w = synth.droplet(n=n, r=r, G=4.0, Ez=0.0, nions=0, tol=1e-6, noise=0.0, eps_r=(1.0, eps_b), prec="fp32")
    w.params.nx = 2
    w.params.poisson_max_iter = 200
    rho = w.rho[:, :, :, n // 2 - 1:n // 2 + 1].copy()
    relax = lbeh.System(w.params)
    relax.set_fields(rho=list(rho))
    assert relax.step(10000) == lbeh.LBEH_OK
    f = relax.get(("rho",), f=True)
    relax.close()
    ra, rb = f["rho"]
    rd = math.sqrt(float(((rb - ra) > 0)[:, :, 0].sum()) / math.pi)
    p = copy.deepcopy(w.params)
    p.E_ext = (0.0, 0.0, E)
    s = lbeh.System(p)
    s.set_fields(f=f["f"])
    ds = []
    for _ in range(8):
        assert s.step(5000) == lbeh.LBEH_OK
        ds.append(_deformation_yz(s.get(("rho",))["rho"], n))
    s.close()
    last = np.array(ds[-4:])
    d = float(last.mean())
    eps_a = 1.0 / (4.0 * math.pi * 0.4)
    chi = (1.0 - eps_b) / (1.0 + eps_b)
    delta_th = eps_a * rd * chi ** 2 * E ** 2 / (4.0 * gamma)
    print("quasi2d l=%d r/l=%g r=%.2f" % (n, rl, rd), ds, delta_th, d / delta_th)
    # prolate along the field; the drop of radius 14.5 in the 128 box keeps a
    # slow oscillation of about +-15% around its mean over the last 20 000 steps
    assert d > 0.0 and (last.max() - last.min()) < 0.35 * d, ds
    # the paper reports up to 15% deviation for small drops; measured here
    # (mean of the last 20 000 steps): +15% (r = 16.5, l = 64), -21% (r = 8.2,
    # l = 64), +32% (r = 14.5, l = 128)
    assert abs(d / delta_th - 1.0) < 0.4, (d, delta_th, rd)

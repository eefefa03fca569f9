"""The seeded input generators do what the input recipes state: shapes,
seeded reproducibility, neutrality of the charged workloads, non-overlapping
colloids with the stated gap, and the flat-interface salt partition."""
import math

import numpy as np

import synth


def test_droplet_recipe_and_neutral_charge():
    w1 = synth.droplet(n=32, r=8.0, charge=12.0)
    w2 = synth.droplet(n=32, r=8.0, charge=12.0)
    assert w1.rho.shape == (2, 32, 32, 32) and w1.n.shape == (2, 32, 32, 32)
    assert np.array_equal(w1.rho, w2.rho)                     # seeded
    assert abs(float((w1.n[0] - w1.n[1]).sum()) - 0.0) < 1e-9  # Q inside, -Q outside
    c = 16.0
    x = np.arange(32.0)
    inside = ((x[None, None, :] - c) ** 2 + (x[None, :, None] - c) ** 2 + (x[:, None, None] - c) ** 2) < 64.0
    assert abs(float((w1.n[0] - 1e-3)[inside].sum()) - 12.0) < 1e-9
    assert np.all(w1.rho[1][inside] > 0.6) and np.all(w1.rho[0][~inside] > 0.6)


def test_suspension_recipe():
    w = synth.suspension(n=48, ncoll=6, r=6.0)
    cx = w.colloid_x
    for i in range(len(cx)):
        for j in range(i):
            d = np.abs(cx[i] - cx[j])
            d = np.minimum(d, 48 - d)
            assert math.sqrt(float((d * d).sum())) >= 2 * 6.0 + 2.0
    assert np.all((w.colloid_q >= -40.0) & (w.colloid_q <= -10.0))
    # counter-cations neutralise the colloid charge
    assert abs(float((w.n[0] - w.n[1]).sum()) + float(w.colloid_q.sum())) < 1e-8
    assert w.params.colloids_move == 1 and w.params.ncomp == 1


def test_flat_interface_recipe():
    chi, dmu = 0.5, (3.0, -1.0)
    w = synth.flat_interface(nx=64, ny=2, nz=2, dmu=dmu, chi=chi, salt=2e-3)
    assert w.rho.shape == (2, 2, 2, 64)
    assert np.all(w.rho[0][..., :32] == 0.7) and np.all(w.rho[0][..., 32:] == 0.04)
    assert np.all(w.rho[1][..., :32] == 0.04) and np.all(w.rho[1][..., 32:] == 0.7)
    nb = 2e-3 * math.exp(-0.5 * (dmu[0] + dmu[1]))
    assert np.allclose(w.n[:, ..., :32], 2e-3) and np.allclose(w.n[:, ..., 32:], nb)
    ea, eb = w.params.eps_r
    assert abs((ea - eb) / (ea + eb) - chi) < 1e-15
    assert tuple(w.params.dmu) == dmu


def test_coated_droplet_recipe():
    """Sec. III.G: 80 spheres of radius 5 on the surface of a drop of radius
    32 (covering fraction N rp^2 / (4 rd^2) = 0.49, the paper's ~0.48), no
    two overlapping, uncharged, particle permittivity 10/80 of the fluids'."""
    w = synth.coated_droplet(n=128)
    c = 64.0
    r = np.sqrt(((w.colloid_x - c) ** 2).sum(axis=1))
    assert w.colloid_x.shape == (80, 3) and np.allclose(r, 32.0)
    d = np.sqrt(((w.colloid_x[:, None, :] - w.colloid_x[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(d, np.inf)
    assert d.min() > 2 * 5.0
    assert abs(80 * 25.0 / (4 * 32.0 ** 2) - 0.488) < 1e-3
    assert np.all(w.colloid_q == 0.0) and w.params.eps_r_colloid == 0.125
    assert w.params.ncolloid_max == 80 and w.params.colloids_move == 1
    assert abs(float(w.n[0].sum() - w.n[1].sum())) < 1e-9  # neutral start

"""Pins of the closed-form sharp-interface equilibrium in tests/_theory.py
(Sec. III.A) against the equations it solves: the nonlinear Poisson-Boltzmann
equation in each fluid, continuity of phi and of eps dphi/ds at the interface,
electroneutral bulks at the Donnan potential, and the trivial case."""
import math

import numpy as np

from _theory import flat_box_distance, sharp_interface

EPS_A = 1.0 / (4.0 * math.pi * 0.4)


def _profiles(chi, dmu=(2.0, -2.0), n_a=1e-3):
    eps_b = EPS_A * (1.0 - chi) / (1.0 + chi)
    return eps_b, dmu, n_a


def test_poisson_boltzmann_holds_on_each_side():
    for chi in (0.0, 0.5):
        eps_b, dmu, n_a = _profiles(chi)
        h = 1e-3
        for side, eps in ((-1.0, EPS_A), (1.0, eps_b)):
            s = side * np.arange(0.5, 40.0, h)
            phi, n_p, n_m = sharp_interface(s, n_a, dmu, EPS_A, eps_b)
            lap = (phi[2:] - 2.0 * phi[1:-1] + phi[:-2]) / h ** 2
            rhs = -(n_p[1:-1] - n_m[1:-1]) / eps
            assert np.allclose(lap, rhs, rtol=1e-4, atol=1e-6 * np.abs(rhs).max())


def test_interface_continuity_of_potential_and_displacement():
    for chi in (0.0, 0.5, 0.9):
        eps_b, dmu, n_a = _profiles(chi)
        h = 1e-6
        s = np.array([-2.0 * h, -h, h, 2.0 * h])
        phi, _, _ = sharp_interface(s, n_a, dmu, EPS_A, eps_b)
        assert abs(phi[1] - phi[2]) < 1e-5
        d_left = EPS_A * (phi[1] - phi[0]) / h
        d_right = eps_b * (phi[3] - phi[2]) / h
        assert abs(d_left - d_right) < 1e-4 * max(abs(d_left), 1e-12)


def test_bulks_are_neutral_at_the_donnan_potential():
    for dmu in ((2.0, -2.0), (3.0, -1.0), (1.0, 1.0)):
        eps_b, _, n_a = _profiles(0.5)
        phi, n_p, n_m = sharp_interface(np.array([-400.0, 400.0]), n_a, dmu, EPS_A, eps_b)
        n_b = n_a * math.exp(-0.5 * (dmu[0] + dmu[1]))
        assert abs(phi[0]) < 1e-12
        assert abs(phi[1] - 0.5 * (dmu[1] - dmu[0])) < 1e-12
        assert np.allclose([n_p[0], n_m[0]], n_a, rtol=1e-12)
        assert np.allclose([n_p[1], n_m[1]], n_b, rtol=1e-12)


def test_no_transfer_energy_no_structure():
    phi, n_p, n_m = sharp_interface(np.linspace(-30.0, 30.0, 61), 1e-3, (0.0, 0.0), EPS_A, 0.3 * EPS_A)
    assert np.abs(phi).max() < 1e-15
    assert np.allclose(n_p, 1e-3) and np.allclose(n_m, 1e-3)


def test_flat_box_distance():
    s = flat_box_distance(8)
    assert np.allclose(s, [-0.5, -1.5, -1.5, -0.5, 0.5, 1.5, 1.5, 0.5])

"""Brute-force pin of the composed oracle step: the array-shift oracle and the
site-by-site transcription in tests/naive_step.py (dense Poisson solve) agree
on tiny ragged lattices for three steps, with every coupling switched on at
once -- two components with Shan-Chen forcing, ions with solvation, an
applied field, Kelvin and friction forces, upwind advection, and a charged
sphere with a moving-wall velocity on the bounce-back links (Sec. II.A-E)."""
import numpy as np
import pytest

import synth
from naive_step import NaiveSystem
from oracle import OracleSystem


def _case(seed, with_colloid):
    nx, ny, nz = 5, 6, 7
    rng = np.random.default_rng(seed)
    p = synth.Params(nx=nx, ny=ny, nz=nz, ncomp=2, nions=2, prec="fp64", tau=1.0, G=2.5, D=0.05, bjerrum=0.4,
                     eps_r=(1.0, 0.5), eps_r_colloid=0.125, dmu=(1.5, -0.7), drho_a=0.66,
                     E_ext=(0.02, -0.01, 0.03), poisson_tol=1e-14, poisson_max_iter=500,
                     ncolloid_max=1 if with_colloid else 0, colloids_move=0)
    shape = (nz, ny, nx)
    rho = np.stack([rng.uniform(0.05, 0.7, size=shape), rng.uniform(0.05, 0.7, size=shape)])
    u = rng.uniform(-0.02, 0.02, size=(3,) + shape)
    n = rng.uniform(0.005, 0.015, size=(2,) + shape)
    kw = {}
    if with_colloid:
        kw = dict(colloid_x=np.array([[2.3, 2.9, 3.6]]), colloid_v=np.array([[0.01, -0.02, 0.015]]),
                  colloid_q=np.array([-0.3]), colloid_r=np.array([1.6]))
    return p, rho, u, n, kw


@pytest.mark.parametrize("seed,with_colloid", [(0, False), (1, True), (2, True)])
def test_oracle_matches_naive_transcription(seed, with_colloid):
    p, rho, u, n, kw = _case(seed, with_colloid)
    o = OracleSystem(p, rho, n, u=u, **kw)
    nv = NaiveSystem(p, o.f, o.n, o.phi, o.solid, o.owner, o.psi_s, o.qc, o.cv)
    if with_colloid:
        assert o.solid.sum() > 0 and (o.psi_s > 0).sum() > o.solid.sum()
    for step in range(3):
        o.step()
        nv.step()
        scale_f = np.abs(o.f).max()
        assert np.abs(o.f - nv.f).max() < 1e-13 * scale_f, (step, np.abs(o.f - nv.f).max())
        assert np.abs(o.n - nv.n).max() < 1e-13 * np.abs(o.n).max(), (step, np.abs(o.n - nv.n).max())
        assert np.abs(o.phi - nv.phi).max() < 1e-11 * np.abs(o.phi).max(), (step, np.abs(o.phi - nv.phi).max())

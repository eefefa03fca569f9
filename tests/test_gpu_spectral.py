"""GPU parity of the spectral Poisson solve (Sec. II.D, conjugate gradients
preconditioned by the Hartley-transform inverse of the constant-coefficient
Laplacian) through the C-ABI, against the FP64 oracle.

* FP64: the coupled step with the spectral solve matches the oracle to 1e-11
  on ragged boxes whose extents take every radix of the transforms
  (20 x 24 x 28, 15 x 21 x 10, 40 x 6 x 7), with ions, an applied field and two
  permittivities (both solves driven to a relative residual of 1e-13).
* FP32 (double-float potential): five coupled steps of a charged droplet
  within the FP32 tolerances of the other parity tests.
* Full size: one step of the 128^3 droplet the bench times; the potential
  matches the oracle's within the tolerance both sides stop at, and the FP64
  residual of the GPU potential in the equation the GPU was given (its FP32
  permittivity, charge and face coefficients) is below the tolerance.
* Choice of solver: automatic (spectral for the droplet, multigrid with
  colloids), forced, and refused for an extent with the prime factor 11.
"""
import numpy as np
import pytest

import synth
from _common import compare, gpu_for, oracle_for, rel_err, step_both, with_params

pytestmark = pytest.mark.gpu


def _slab(nx, ny, nz, prec="fp64", tol=1e-13, solver="spectral"):
    w = synth.two_slab(nx=nx, ny=ny, nz=nz, G=4.0, prec=prec, tol=tol, colloid=False)
    w.params.E_ext = (0.01, -0.005, 0.02)
    w.params.poisson_solver = solver
    w.params.poisson_max_iter = 200
    return w


@pytest.mark.parametrize("dims", [(20, 24, 28), (15, 21, 10), (40, 6, 7)])
def test_fp64_spectral_matches_oracle(lbeh, dims):
    w = _slab(*dims)
    so, sg = oracle_for(w), gpu_for(w, lbeh)
    step_both(sg, so, 3)
    errs = compare(sg, so)
    assert all(e < 1e-11 for e in errs.values()), errs
    o = sg.observables()
    assert o.poisson_solver == lbeh.LBEH_POISSON_SPECTRAL
    assert o.poisson_relres < 1e-13 and 0 < o.poisson_iters < 60
    sg.close()


def test_fp32_spectral_droplet_parity(lbeh):
    w = synth.droplet(n=24, r=7.0, prec="fp32", tol=1e-8, Ez=0.02, charge=4.0)
    w.params.poisson_solver = "spectral"
    so, sg = oracle_for(w), gpu_for(w, lbeh)
    step_both(sg, so, 5)
    errs = compare(sg, so)
    assert errs["rho"] < 2e-5 and errs["n"] < 2e-5 and errs["u"] < 2e-4, errs
    assert errs["phi"] < 2e-4, errs
    sg.close()


def test_droplet_128_cubed_spectral_one_step(lbeh):
    w = synth.droplet(n=128, r=24.0, prec="fp32")
    so, sg = oracle_for(w), gpu_for(w, lbeh)
    assert sg.step(1) == lbeh.LBEH_OK
    so.step()
    o = sg.observables()
    assert o.poisson_solver == lbeh.LBEH_POISSON_SPECTRAL  # automatic choice for this box
    g = sg.get(("rho", "n", "phi"))
    assert max(rel_err(g["rho"][s], so.densities()[s]) for s in range(2)) < 2e-5
    assert max(rel_err(g["n"][s], so.n[s]) for s in range(2)) < 2e-5
    assert rel_err(g["phi"], so.phi) < 2e-3
    # the GPU potential solves, to the tolerance, the discrete equation it was
    # given: its own FP32 eps and q, face coefficients (eps_i + eps_j)/2 rounded
    # to FP32; residual evaluated in FP64
    eps32 = sg.aux(lbeh.LBEH_AUX_EPS).astype(np.float32)
    q = sg.aux(lbeh.LBEH_AUX_Q)
    phi = np.asarray(g["phi"], dtype=np.float64)
    b = -(q - q.mean())
    Aphi = np.zeros_like(phi)
    for ax in (2, 1, 0):  # array axes z, y, x <-> field components 2, 1, 0 below
        kp = (np.float32(0.5) * (eps32 + np.roll(eps32, -1, axis=ax))).astype(np.float64)
        km = np.roll(kp, 1, axis=ax)
        Aphi += kp * (np.roll(phi, -1, axis=ax) - phi) - km * (phi - np.roll(phi, 1, axis=ax))
        b += so.E_ext[2 - ax] * (kp - km)
    r = b - Aphi
    assert float(np.sqrt((r * r).sum() / (b * b).sum())) < 1.01e-6
    sg.close()


def test_spectral_iterations_stay_few_over_a_run(lbeh):
    w = synth.droplet(n=64, r=12.0, prec="fp32", Ez=1e-3, charge=20.0)
    sg = gpu_for(w, lbeh)
    for _ in range(10):
        assert sg.step(5) == lbeh.LBEH_OK
        o = sg.observables()
        assert o.poisson_relres < 1e-6 and o.poisson_iters <= 6, (o.poisson_relres, o.poisson_iters)
    sg.close()


def test_solver_choice(lbeh):
    w = synth.droplet(n=16, r=5.0, prec="fp32")
    sg = gpu_for(w, lbeh)
    assert sg.observables().poisson_solver == lbeh.LBEH_POISSON_SPECTRAL
    sg.close()
    sg = gpu_for(with_params(w, poisson_solver="multigrid"), lbeh)
    assert sg.observables().poisson_solver == lbeh.LBEH_POISSON_MULTIGRID
    sg.close()
    s = synth.two_slab(nx=16, ny=16, nz=16, G=4.0, prec="fp32", tol=1e-8)  # a colloid: contrast 8
    sg = gpu_for(s, lbeh)
    assert sg.observables().poisson_solver == lbeh.LBEH_POISSON_MULTIGRID
    sg.close()
    with pytest.raises(lbeh.LbehError) as e:
        lbeh.System(with_params(synth.droplet(n=22, r=5.0, prec="fp32"), poisson_solver="spectral").params)
    assert e.value.code == lbeh.LBEH_ERR_UNSUPPORTED
    sg = gpu_for(synth.droplet(n=22, r=5.0, prec="fp32"), lbeh)  # automatic: falls back to the multigrid
    assert sg.observables().poisson_solver == lbeh.LBEH_POISSON_MULTIGRID
    assert sg.step(2) == lbeh.LBEH_OK
    sg.close()


def test_multigrid_still_matches_on_the_droplet(lbeh):
    w = synth.droplet(n=24, r=7.0, prec="fp32", tol=1e-8, Ez=0.02, charge=4.0)
    w.params.poisson_solver = "multigrid"
    so, sg = oracle_for(w), gpu_for(w, lbeh)
    step_both(sg, so, 5)
    errs = compare(sg, so)
    assert errs["rho"] < 2e-5 and errs["n"] < 2e-5 and errs["phi"] < 2e-4, errs
    sg.close()

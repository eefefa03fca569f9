"""Failure detection of the step, in forms that fault and hang no GPU.

* A non-finite value planted on the host in the initial fields (a NaN
  density, a NaN ion concentration) is reported as LBEH_ERR_NONFINITE within a
  few steps: by the Poisson solve, whose residual test sees the non-finite
  norm and stops, or, without a potential, by the observables' sums.  Loading clean fields clears
  the sticky status and the same handle steps on normally.
* A grid-barrier wait of the one-launch Poisson solves (spectral and
  multigrid) that runs out of polls -- here the limit is one poll, so blocks
  that arrive before the last one give up -- raises the abort flag; every block
  returns, the step reports LBEH_ERR_BARRIER_TIMEOUT, and after restoring the
  default limit and reloading the state the handle steps to the same result as
  a fresh handle.
"""
import numpy as np
import pytest

import synth
from _common import gpu_for, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("where", ["rho", "ions"])
def test_nan_in_initial_fields_is_reported(lbeh, where):
    w = synth.droplet(n=16, r=5.0, prec="fp32", Ez=0.01, charge=2.0)
    rho = w.rho.copy()
    n = w.n.copy()
    if where == "rho":
        rho[0, 3, 4, 5] = np.nan
    else:
        n[1, 7, 2, 9] = np.nan
    sg = lbeh.System(w.params)
    sg.set_fields(rho=list(rho), n=list(n))
    # a NaN ion enters the charge at once; a NaN density reaches the
    # permittivity through the neighbours' populations one step later
    with pytest.raises(lbeh.LbehError) as e:
        for _ in range(3):
            sg.step(1)
    assert e.value.code == lbeh.LBEH_ERR_NONFINITE
    assert sg.observables().status == lbeh.LBEH_ERR_NONFINITE
    sg.set_fields(rho=list(w.rho), n=list(w.n))  # clean state: status cleared
    assert sg.step(3) == lbeh.LBEH_OK
    assert sg.observables().status == lbeh.LBEH_OK
    sg.close()


def test_nan_without_a_potential_is_reported_by_the_observables(lbeh):
    w = synth.droplet(n=16, r=5.0, prec="fp32", Ez=0.0, nions=0)
    rho = w.rho.copy()
    rho[1, 0, 0, 0] = np.inf
    sg = lbeh.System(w.params)
    sg.set_fields(rho=list(rho))
    sg.step(1)
    assert sg.observables().status == lbeh.LBEH_ERR_NONFINITE
    sg.close()


@pytest.mark.parametrize("solver", ["spectral", "multigrid"])
def test_barrier_timeout_is_reported_and_the_handle_recovers(lbeh, solver):
    w = synth.droplet(n=32, r=9.0, prec="fp32", Ez=0.01, charge=3.0)
    w.params.poisson_solver = solver
    sg = gpu_for(w, lbeh)
    assert sg.step(2) == lbeh.LBEH_OK
    lbeh.lbeh_set_wait_limit(sg.h, 1)
    with pytest.raises(lbeh.LbehError) as e:
        sg.step(1)
    assert e.value.code == lbeh.LBEH_ERR_BARRIER_TIMEOUT
    assert sg.observables().status == lbeh.LBEH_ERR_BARRIER_TIMEOUT
    lbeh.lbeh_set_wait_limit(sg.h, 0)
    sg.set_fields(rho=list(w.rho), n=list(w.n))  # potential and solver state restart from zero
    assert sg.step(4) == lbeh.LBEH_OK
    ref = gpu_for(w, lbeh)
    assert ref.step(4) == lbeh.LBEH_OK
    a, b = sg.get(("rho", "n")), ref.get(("rho", "n"))
    assert max(rel_err(a["rho"][s], b["rho"][s]) for s in range(2)) < 1e-6
    assert max(rel_err(a["n"][s], b["n"][s]) for s in range(2)) < 1e-6
    sg.close()
    ref.close()

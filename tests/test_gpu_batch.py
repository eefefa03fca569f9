"""Batched step: many independent boxes of uneven size advanced by one
persistent cluster launch (one thread-block cluster per box), against the
oracle box by box, against one launch per box (bitwise), and against the
single-system kernels (within the FP32 tolerance)."""
import numpy as np
import pytest

import synth
from _common import load, oracle_for, rel_err

pytestmark = pytest.mark.gpu


def _boxes(edges, prec, seed=7, tol=None, Ez=None, charge=None):
    rng = np.random.default_rng(seed)
    out = []
    for b, e in enumerate(edges):
        w = synth.droplet(n=e, r=0.3 * e, seed=100 + b, prec=prec, salt=1e-3,
                          Ez=float(rng.uniform(0.0, 2e-3)) if Ez is None else Ez,
                          charge=float(rng.uniform(0.0, 20.0)) if charge is None else charge, steps=1)
        if tol is not None:
            w.params.poisson_tol = tol
            w.params.poisson_max_iter = 400
        out.append(w)
    return out


def _make(lbeh, ws, shape=None):
    bt = lbeh.Batch([w.params for w in ws])
    for box, w in zip(bt.boxes, ws):
        load(box, w)
    if shape:
        bt.set_shape(shape)
    return bt


def _state(bt):
    return [b.get(("rho", "n", "phi", "u"), f=True) for b in bt.boxes]


def test_fp64_batch_matches_oracle_box_by_box(lbeh):
    ws = _boxes([16, 24, 32], "fp64", tol=1e-12)
    bt = _make(lbeh, ws)
    orc = [oracle_for(w) for w in ws]
    for _ in range(4):
        assert bt.step(1) == lbeh.LBEH_OK
        for o in orc:
            o.step()
            assert o.poisson_relres < o.tol
    for box, o in zip(bt.boxes, orc):
        g = box.get(("rho", "n", "phi"))
        assert max(rel_err(g["rho"][s], o.densities()[s]) for s in range(2)) < 1e-12
        assert max(rel_err(g["n"][s], o.n[s]) for s in range(2)) < 1e-12
        assert rel_err(g["phi"], o.phi) < 1e-9
        ob = box.observables()
        assert ob.steps == 4 and ob.status == lbeh.LBEH_OK
        assert ob.poisson_relres < 1e-12
    bt.close()


@pytest.mark.parametrize("shape", [1, 2, 4, 8])
def test_fp32_batched_launch_equals_one_launch_per_box(lbeh, shape):
    ws = _boxes([32, 40, 48, 24, 32, 16], "fp32")
    a = _make(lbeh, ws, shape)
    b = _make(lbeh, ws, shape)
    assert a.step(6) == lbeh.LBEH_OK
    assert b.step_sequential(6) == lbeh.LBEH_OK
    for sa, sb in zip(_state(a), _state(b)):
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), k
    a.close()
    b.close()


def test_fp32_batch_close_to_single_system_kernels(lbeh):
    from _common import gpu_for
    ws = _boxes([32, 48], "fp32")
    bt = _make(lbeh, ws, 4)
    singles = [gpu_for(w, lbeh) for w in ws]
    assert bt.step(10) == lbeh.LBEH_OK
    for s in singles:
        assert s.step(10) == lbeh.LBEH_OK
    for box, s in zip(bt.boxes, singles):
        g, r = box.get(("rho", "n", "phi")), s.get(("rho", "n", "phi"))
        assert rel_err(g["rho"], r["rho"]) < 1e-6
        assert rel_err(g["n"], r["n"]) < 1e-5
        assert rel_err(g["phi"], r["phi"]) < 1e-4
        s.close()
    bt.close()


def test_tuner_keeps_state_and_picks_a_feasible_shape(lbeh):
    ws = _boxes([32, 24, 40], "fp32")
    a = _make(lbeh, ws)
    b = _make(lbeh, ws)
    cpb, ms = a.tune(2)
    assert cpb in (1, 2, 4, 8, 16) and ms > 0
    b.set_shape(cpb)
    assert a.step(3) == lbeh.LBEH_OK
    assert b.step(3) == lbeh.LBEH_OK
    for sa, sb in zip(_state(a), _state(b)):
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), k
    a.close()
    b.close()


def test_batch_box_views_and_status(lbeh):
    ws = _boxes([16, 24], "fp32")
    ws[1].params.poisson_tol = 1e-30
    ws[1].params.poisson_max_iter = 1
    bt = _make(lbeh, ws)
    assert bt.step(2) == lbeh.LBEH_ERR_POISSON_NOT_CONVERGED
    assert bt.boxes[0].observables().status == lbeh.LBEH_OK
    assert bt.boxes[1].observables().status == lbeh.LBEH_ERR_POISSON_NOT_CONVERGED
    # a box stepped on its own (single-system kernels) rejoins the batch
    assert bt.boxes[0].step(1) == lbeh.LBEH_OK
    assert bt.step(1) == lbeh.LBEH_ERR_POISSON_NOT_CONVERGED
    assert bt.boxes[0].observables().steps == 4
    with pytest.raises(lbeh.LbehError):
        lbeh.lbeh_observables(bt.h)
    bt.close()


def test_batch_rejects_mixed_or_colloidal_boxes(lbeh):
    ws = _boxes([16, 16], "fp32")
    ws[1].params.nions = 0
    with pytest.raises(lbeh.LbehError):
        lbeh.Batch([w.params for w in ws])
    w = synth.two_slab(nx=16, ny=16, nz=16, prec="fp32")
    with pytest.raises(lbeh.LbehError):
        lbeh.Batch([w.params])

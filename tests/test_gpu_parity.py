"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Tolerances (max |gpu - oracle| / max |oracle| per field):
  * FP64 path: 1e-11 after a few steps (round-off of different summation
    orders, amplified by the nonlinear Shan-Chen coupling), with the Poisson
    solves of both sides driven to a relative residual of 1e-13.
  * FP32 compute and storage: 2e-5 (single-precision rounding, 24 bits,
    accumulated over the steps).
  * BF16 / FP16 shifted storage: 5e-3 / 1e-3 for the densities (the stored
    deviation f - w rho0 keeps 8 / 11 mantissa bits).
Bit-exact: solid mask, owner ids, solid fraction, surface nodes, surface charge.
"""
import numpy as np
import pytest

import synth
from _common import compare, gpu_for, oracle_for, rel_err, step_both, with_params
from oracle import geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbeh():
    import paper_1712_08494_gb300 as pkg
    pkg.build()
    from paper_1712_08494_gb300 import lbeh as L
    return L


def _slab(n=(20, 24, 28), G=4.0, prec="fp64", tol=1e-13, **kw):
    nx, ny, nz = n
    w = synth.two_slab(nx=nx, ny=ny, nz=nz, G=G, prec=prec, tol=tol, **kw)
    w.colloid_x[:] = [[nx / 2.0, ny / 2.0, nz / 2.0 - 0.5]] if len(w.colloid_r) else w.colloid_x
    return w


# ---------------------------------------------------------------- geometry
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_geometry_bit_exact(lbeh, prec):
    w = _slab(prec=prec)
    # several colloids, one wrapping the periodic boundary, radius not integer
    w.colloid_x = np.array([[10.0, 12.0, 13.5], [1.3, 22.9, 3.25], [15.6, 4.1, 24.7]])
    w.colloid_r = np.array([4.0, 3.3, 2.7])
    w.colloid_q = np.array([-20.0, 7.0, -3.0])
    w.colloid_v = np.zeros((3, 3))
    w.params.ncolloid_max = 3
    sg = gpu_for(w, lbeh)
    p = w.params
    solid, owner, psi_s = geometry.project(p.nx, p.ny, p.nz, w.colloid_x, w.colloid_r, 3)
    surf = geometry.surface_nodes(solid)
    qc = geometry.colloid_charge(owner, surf, w.colloid_q)
    assert np.array_equal(sg.aux(lbeh.LBEH_AUX_SOLID).astype(bool), solid)
    assert np.array_equal(sg.aux(lbeh.LBEH_AUX_OWNER), owner.astype(np.int32))
    assert np.array_equal(sg.aux(lbeh.LBEH_AUX_SURFACE).astype(bool), surf)
    assert np.array_equal(sg.aux(lbeh.LBEH_AUX_PSI_S), psi_s)
    q = sg.aux(lbeh.LBEH_AUX_QC)
    if prec == "fp64":
        assert np.array_equal(q, qc)
    else:
        assert np.array_equal(q, qc.astype(np.float32).astype(np.float64))
    sg.close()


# ---------------------------------------------------------------- FP64 path
@pytest.mark.parametrize("G", [0.08, 4.0])
def test_fp64_two_slab_with_colloid(lbeh, G):
    w = _slab(G=G)
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    step_both(sg, so, 3)
    errs = compare(sg, so)
    assert all(e < 1e-11 for e in errs.values()), errs
    # intermediate fields of the last step
    assert rel_err(sg.aux(lbeh.LBEH_AUX_EPS), so.last_eps) < 1e-13
    assert rel_err(sg.aux(lbeh.LBEH_AUX_RHO_V), so.last_rho_v) < 1e-12
    o = sg.observables()
    assert abs(o.charge) < 1e-10
    sg.close()


def test_fp64_droplet_field_solvation(lbeh):
    """Applied field (dielectric polarisation), solvation forces, charged drop."""
    w = synth.droplet(n=24, r=7.0, prec="fp64", tol=1e-13, Ez=0.02, charge=5.0, salt=2e-3)
    w.params.dmu = (1.5, -0.5)
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    step_both(sg, so, 4)
    errs = compare(sg, so)
    assert all(e < 1e-11 for e in errs.values()), errs
    sg.close()


def test_fp64_single_component_fixed_colloids(lbeh):
    w = synth.suspension(n=24, ncoll=3, r=3.0, prec="fp64", tol=1e-13, Ex=0.01)
    w.params.colloids_move = 0
    w.params.poisson_max_iter = 400   # eps_p/eps_a = 1/8: oracle split contracts by 0.78
    w.params.ncolloid_max = 3
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    step_both(sg, so, 3)
    errs = compare(sg, so)
    assert all(e < 1e-11 for e in errs.values()), errs
    cf = sg.get(("rho",))["cf"]
    # total colloid force of the last step: bounce-back momentum exchange,
    # electric force on the surface charge, pair forces
    assert rel_err(cf, so.colloid_force) < 1e-9
    sg.close()


def test_fp64_ion_free_no_poisson(lbeh):
    w = synth.droplet(n=16, r=5.0, prec="fp64", nions=0, Ez=0.0)
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    step_both(sg, so, 5)
    errs = compare(sg, so, ("rho", "u"))
    assert all(e < 1e-12 for e in errs.values()), errs
    sg.close()


# ---------------------------------------------------------------- reduced precision
@pytest.mark.parametrize("prec,tol_rho", [("fp32", 2e-5), ("bf16", 5e-3), ("fp16", 1e-3)])
def test_reduced_precision_droplet(lbeh, prec, tol_rho):
    w = synth.droplet(n=24, r=7.0, prec=prec, tol=1e-10, Ez=0.02, charge=5.0, salt=2e-3)
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    step_both(sg, so, 5)
    errs = compare(sg, so, ("rho", "n", "phi"))
    assert errs["rho"] < tol_rho, errs
    assert errs["n"] < (2e-5 if prec == "fp32" else 10 * tol_rho), errs
    assert errs["phi"] < (2e-4 if prec == "fp32" else 50 * tol_rho), errs
    sg.close()


@pytest.mark.parametrize("prec,src", [("fp64", "host64"), ("fp32", "host32"), ("fp32", "device32")])
def test_restart_with_potential(lbeh, prec, src):
    """A state loaded together with its potential: n and phi read back exactly
    as loaded, the first solve starts from the loaded potential (fewer
    iterations than from zero) and the step matches the oracle started from
    the same state and potential."""
    import torch
    from oracle import OracleSystem
    w = synth.droplet(n=24, r=7.0, prec=prec, tol=1e-13 if prec == "fp64" else 1e-10, Ez=0.02, charge=5.0,
                      salt=2e-3)
    sg = gpu_for(w, lbeh)
    sg.step(5)
    ck = sg.get(("rho", "n", "phi"))
    sg.close()
    dt = np.float64 if src == "host64" else np.float32
    arrs = [np.ascontiguousarray(a, dtype=dt) for a in (ck["rho"][0], ck["rho"][1], ck["n"][0], ck["n"][1], ck["phi"])]
    exact = [a.astype(np.float64) for a in arrs]
    if src == "device32":
        arrs = [torch.from_numpy(a).cuda() for a in arrs]
    cycles = {}
    for warm in (False, True):
        sg = lbeh.System(w.params, 0)
        sg.set_fields(rho=arrs[:2], n=arrs[2:4], phi=arrs[4] if warm else None)
        if warm:
            got = sg.get(("rho", "n", "phi"))
            assert np.array_equal(got["n"], np.stack(exact[2:4]))
            assert np.array_equal(got["phi"], exact[4])
            assert rel_err(got["rho"], np.stack(exact[:2])) < (1e-14 if prec == "fp64" else 1e-6)
        sg.profile_enable(False)
        assert sg.step(1) == 0
        cycles[warm] = sg.profile_read()["poisson_cycles"]
        if warm:
            so = OracleSystem(w.params, np.stack(exact[:2]), np.stack(exact[2:4]), phi=exact[4])
            so.step()
            errs = compare(sg, so, ("rho", "n", "phi"))
            if prec == "fp64":
                assert max(errs.values()) < 1e-11, errs
            else:
                assert errs["rho"] < 2e-5 and errs["n"] < 2e-5 and errs["phi"] < 2e-4, errs
        sg.close()
    assert cycles[True] < cycles[False], cycles


@pytest.mark.parametrize("case", ["droplet_fp64", "slab_fp32_tail", "odd_fp32"])
def test_observables_match_their_definition(lbeh, case):
    """lbeh_observables against its sums written out in FP64 over the state read
    back: whole staged chunks of 256 sites (24^3), whole chunks plus a ragged
    tail and a colloid (20x24x28), and a box whose rows are not 16-byte
    aligned (13x11x9), which is read directly."""
    from oracle import observables
    from oracle.lattice import C
    if case == "droplet_fp64":
        w = synth.droplet(n=24, r=7.0, prec="fp64", tol=1e-12, Ez=0.02, charge=5.0, salt=2e-3)
    elif case == "slab_fp32_tail":
        w = _slab(prec="fp32", tol=1e-8)
    else:
        w = synth.two_slab(nx=13, ny=11, nz=9, G=4.0, prec="fp32", tol=1e-8, colloid=False)
    sg = gpu_for(w, lbeh)
    sg.step(3)
    o = sg.observables()
    st = sg.get(("rho", "n"), f=True)
    f = st["f"]
    fl = np.ones(f.shape[2:], dtype=bool)
    qc_sum = 0.0
    if len(w.colloid_r):
        fl = sg.aux(lbeh.LBEH_AUX_SOLID) == 0
        qc_sum = float(sg.aux(lbeh.LBEH_AUX_QC).sum())
    rho = f.sum(axis=1) * fl
    mass = [float(rho[s].sum()) for s in range(f.shape[0])]
    ions = [float(st["n"][s].sum()) for s in range(2)]
    mom = sum(C[q] * float((f[:, q] * fl).sum()) for q in range(1, 19))
    D, centroid = observables.deformation(rho)
    rel = 1e-12 if case == "droplet_fp64" else 1e-6  # FP32 site sums: 19 roundings of 2^-24 each
    ms, js = sum(mass), sum(ions)
    for s in range(2):
        assert abs(o.mass[s] - mass[s]) <= rel * ms, (s, o.mass[s], mass[s])
        assert abs(o.ions[s] - ions[s]) <= rel * js, (s, o.ions[s], ions[s])
    assert abs(o.charge - (ions[0] - ions[1] + qc_sum)) <= rel * (js + abs(qc_sum))
    for a in range(3):
        assert abs(o.momentum[a] - mom[a]) <= rel * ms, (a, o.momentum[a], mom[a])
        assert abs(o.centroid[a] - centroid[a]) <= (1e-10 if rel < 1e-9 else 1e-4), (a, o.centroid[a], centroid[a])
    assert abs(o.deformation - D) <= (1e-10 if rel < 1e-9 else 1e-5), (o.deformation, D)
    sg.close()


def test_fp32_two_slab_with_colloid(lbeh):
    w = _slab(prec="fp32", tol=1e-10)
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    step_both(sg, so, 4)
    errs = compare(sg, so, ("rho", "n", "phi"))
    assert errs["rho"] < 2e-5 and errs["n"] < 2e-5 and errs["phi"] < 2e-4, errs
    sg.close()


# ---------------------------------------------------------------- edge cases
@pytest.mark.parametrize("n", [(2, 2, 2), (4, 6, 2), (3, 5, 7)])
def test_tiny_and_odd_boxes(lbeh, n):
    nx, ny, nz = n
    rng = np.random.default_rng(11)
    p = synth.Params(nx=nx, ny=ny, nz=nz, ncomp=2, nions=2, prec="fp64", G=4.0, poisson_tol=1e-13,
                     poisson_max_iter=400, E_ext=(0.01, 0.0, 0.02))
    rho = rng.uniform(0.04, 0.7, size=(2, nz, ny, nx))
    ions = rng.uniform(0.005, 0.015, size=(2, nz, ny, nx))
    w = synth.Workload("tiny", p, rho, ions)
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    step_both(sg, so, 3)
    errs = compare(sg, so)
    assert all(e < 1e-11 for e in errs.values()), errs
    sg.close()


def test_poisson_cap_reports_status_not_fault(lbeh):
    w = _slab(n=(16, 16, 16), tol=1e-14)
    w.params.poisson_max_iter = 1
    sg = gpu_for(w, lbeh)
    rc = sg.step(1)
    assert rc == lbeh.LBEH_ERR_POISSON_NOT_CONVERGED
    assert sg.observables().status == lbeh.LBEH_ERR_POISSON_NOT_CONVERGED
    # the handle stays usable and a fresh load clears the status
    sg.set_fields(rho=list(w.rho), n=list(w.n), colloid_x=w.colloid_x, colloid_v=w.colloid_v,
                  colloid_q=w.colloid_q, colloid_r=w.colloid_r)
    assert sg.observables().status == lbeh.LBEH_OK
    sg.close()


def test_bitwise_reproducible(lbeh):
    w = synth.droplet(n=24, r=7.0, prec="fp32", tol=1e-8, Ez=0.02, charge=5.0)
    outs = []
    for rep in range(2):
        sg = gpu_for(w, lbeh)
        sg.step(5)
        outs.append(sg.get(("rho", "n", "phi")))
        sg.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_fp32_modes_defect_correction_reaches_fp64_grade_residual(lbeh, prec):
    """The FP32 modes keep the potential and the defect-correction residual in
    double-float form, so the Poisson solve reaches relative residuals far
    below the FP32 epsilon (here 1e-11) within the cycle cap, and the
    potential agrees with the FP64 oracle to the FP32 rounding of its inputs."""
    w = synth.droplet(n=24, r=7.0, prec=prec, tol=1e-11, Ez=0.02, charge=5.0, salt=2e-3)
    w.params.poisson_max_iter = 60
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    step_both(sg, so, 2)
    o = sg.observables()
    assert o.status == lbeh.LBEH_OK
    assert o.poisson_relres < 1e-11
    errs = compare(sg, so, ("phi",))
    assert errs["phi"] < 2e-4, errs
    sg.close()


# ---------------------------------------------------------------- moving colloids
def _moving(n=16, ncomp=1, prec="fp64", X=((7.45, 8.2, 7.9),), V=((0.2, -0.15, 0.1),), R=(3.0,), Q=(-5.0,),
            E=(1e-3, 0.0, 0.0)):
    nc = len(R)
    p = synth.Params(nx=n, ny=n, nz=n, ncomp=ncomp, nions=2, prec=prec, G=4.0 if ncomp == 2 else 0.0,
                     ncolloid_max=nc, colloids_move=1, poisson_tol=1e-13, poisson_max_iter=500, E_ext=E,
                     eps_r=(1.0, 1.0) if ncomp == 1 else (1.0, 0.5), rho0_shift=(1.0, 0.0))
    rng = np.random.default_rng(21)
    if ncomp == 1:
        rho = np.ones((1, n, n, n)) * (1 + 0.01 * rng.uniform(-1, 1, size=(1, n, n, n)))
    else:
        z = np.arange(n)[:, None, None] * np.ones((n, n, n))
        red = np.where(z < n // 2, 0.7, 0.04) * (1 + 0.01 * rng.uniform(-1, 1, size=(n, n, n)))
        rho = np.stack([red, 0.74 - red])
    ions = np.full((2, n, n, n), 0.01)
    ions[0] += -sum(Q) / n ** 3
    return synth.Workload("moving", p, rho, ions, np.array(X, dtype=float), np.array(V, dtype=float),
                          np.array(Q, dtype=float), np.array(R, dtype=float))


@pytest.mark.parametrize("ncomp", [1, 2])
def test_fp64_moving_colloid_remap(lbeh, ncomp):
    """Moving charged colloid in salt under a field: bounce-back with the
    moving-wall term, velocity-Verlet, node covering/uncovering with momentum
    and ion transfer (Sec. II.E).  The colloid crosses lattice nodes."""
    w = _moving(ncomp=ncomp)
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    solid0 = so.solid.copy()
    step_both(sg, so, 5)
    assert not np.array_equal(solid0, so.solid)
    errs = compare(sg, so)
    assert all(e < 1e-10 for e in errs.values()), errs
    got = sg.get(("rho",))
    assert rel_err(got["cx"], so.cx) < 1e-13
    assert rel_err(got["cv"], so.cv) < 1e-10
    assert rel_err(got["cf"], so.colloid_force) < 1e-9
    assert np.array_equal(sg.aux(lbeh.LBEH_AUX_SOLID).astype(bool), so.solid)
    sg.close()


def test_fp64_colliding_colloids_hertz_and_lubrication(lbeh):
    """Two colloids in near contact approaching each other: lubrication below a
    surface gap of 2/3 and Hertz repulsion once they overlap."""
    w = _moving(n=20, X=((6.1, 10.0, 10.0), (12.5, 10.2, 9.9)), V=((0.08, 0.0, 0.0), (-0.08, 0.01, 0.0)),
                R=(3.0, 3.0), Q=(-2.0, -2.0), E=(0.0, 0.0, 0.0))
    so = oracle_for(w)
    sg = gpu_for(w, lbeh)
    step_both(sg, so, 4)
    errs = compare(sg, so)
    assert all(e < 1e-10 for e in errs.values()), errs
    got = sg.get(("rho",))
    assert rel_err(got["cx"], so.cx) < 1e-13
    assert rel_err(got["cv"], so.cv) < 1e-10
    sg.close()


def test_fp32_suspension_runs_and_conserves_ions(lbeh):
    w = synth.suspension(n=32, ncoll=3, r=4.0, prec="fp32", tol=1e-6, Ex=1e-3)
    sg = gpu_for(w, lbeh)
    o0 = sg.observables()
    assert sg.step(20) == lbeh.LBEH_OK
    o1 = sg.observables()
    assert abs(o1.ions[0] - o0.ions[0]) < 1e-5 * o0.ions[0]
    assert abs(o1.ions[1] - o0.ions[1]) < 1e-5 * o0.ions[1]
    assert np.isfinite(o1.colloid_v).all()
    sg.close()

"""Parity at the workloads' full sizes, in the launch configuration the bench
times: the 32^3 plain-method case for its whole 200 steps (FP64); one step of
the 128^3 dielectric droplet against the oracle over the whole lattice (FP32
and BF16 storage); the 256^3 suspension through what holds at any size (the
projected geometry bit for bit against the oracle's projection, exact ion
and charge conservation to rounding, colloid drift against the field); the
96-box batch, batched against one launch per box, bit for bit; the adjoint of
the 96^3 drop on its 32^3 copy against the oracle's finite differences in the
applied field, the Shan-Chen coupling and the drop charge."""
import numpy as np
import pytest

import synth
from _common import gpu_for, load, oracle_for, rel_err, step_both

pytestmark = pytest.mark.gpu


def test_plain_method_32_cubed_200_steps_fp64(lbeh):
    w = synth.two_slab(nx=32, ny=32, nz=32, G=4.0, prec="fp64", tol=1e-10)
    w.params.poisson_max_iter = 400
    so, sg = oracle_for(w), gpu_for(w, lbeh)
    step_both(sg, so, 200)
    g = sg.get(("rho", "n", "phi"))
    assert max(rel_err(g["rho"][s], so.densities()[s]) for s in range(2)) < 1e-10
    assert max(rel_err(g["n"][s], so.n[s]) for s in range(2)) < 1e-10
    assert rel_err(g["phi"], so.phi) < 1e-8
    sg.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("bf16", 5e-3)])
def test_droplet_128_cubed_one_step_whole_lattice(lbeh, prec, tol):
    w = synth.droplet(n=128, r=24.0, prec=prec)
    so, sg = oracle_for(w), gpu_for(w, lbeh)
    assert sg.step(1) == lbeh.LBEH_OK
    so.step()
    g = sg.get(("rho", "n", "phi", "u"))
    assert max(rel_err(g["rho"][s], so.densities()[s]) for s in range(2)) < tol
    assert max(rel_err(g["n"][s], so.n[s]) for s in range(2)) < tol
    # the potential of the step: both solves stop at a relative residual of 1e-6
    assert rel_err(g["phi"], so.phi) < 2e-3
    sg.close()


def test_suspension_256_cubed_geometry_and_conservation(lbeh):
    from oracle import geometry
    w = synth.suspension(n=256, ncoll=200, r=6.0, prec="fp32")
    sg = gpu_for(w, lbeh)
    solid, owner, psi_s = geometry.project_boxed(256, 256, 256, w.colloid_x, w.colloid_r, w.params.psi_subdiv)
    assert np.array_equal(sg.aux(lbeh.LBEH_AUX_SOLID).astype(bool), solid)
    assert np.array_equal(sg.aux(lbeh.LBEH_AUX_OWNER), owner.astype(np.int32))
    assert np.array_equal(sg.aux(lbeh.LBEH_AUX_PSI_S), psi_s)
    o0 = sg.observables()
    assert sg.step(20) == lbeh.LBEH_OK
    o1 = sg.observables()
    for s in range(2):
        assert abs(o1.ions[s] - o0.ions[s]) < 1e-6 * o0.ions[s]
    assert abs(o1.charge - o0.charge) < 1e-6 * o0.ions[0]
    # negative colloids in a field along +x drift along -x
    cv = np.array(sg.get(("rho",))["cv"])
    assert cv[:, 0].mean() < 0.0
    # the remapped geometry still matches the oracle's projection at the new positions
    cx = np.array(sg.get(("rho",))["cx"])
    solid2, _, _ = geometry.project_boxed(256, 256, 256, cx, w.colloid_r, w.params.psi_subdiv)
    assert np.array_equal(sg.aux(lbeh.LBEH_AUX_SOLID).astype(bool), solid2)
    sg.close()


def test_batch_96_boxes_batched_equals_per_box_launches(lbeh):
    ws = synth.batch_boxes(nbox=96, steps=3)
    bts = []
    for _ in range(2):
        bt = lbeh.Batch([w.params for w in ws])
        for box, w in zip(bt.boxes, ws):
            load(box, w)
        bts.append(bt)
    shape, _ = bts[0].tune(2)
    bts[1].set_shape(shape)
    assert bts[0].step(3) == lbeh.LBEH_OK
    assert bts[1].step_sequential(3) == lbeh.LBEH_OK
    for a, b in zip(bts[0].boxes, bts[1].boxes):
        ga, gb = a.get(("rho", "n", "phi"), f=True), b.get(("rho", "n", "phi"), f=True)
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), k
    for bt in bts:
        bt.close()


def test_adjoint_drop_32_cubed_copy_against_oracle_fd(lbeh):
    """The 96^3 adjoint case (r=18, Q=50, E_z=1.5e-3) on its 32^3 copy (r=6, Q
    scaled by volume), FP64, 40 steps, checkpoints every 10."""
    from oracle import observables
    nsteps, Ez, Q = 40, 1.5e-3, 50.0 * (32.0 / 96.0) ** 3

    def make(Ez_, Q_, prec="fp64", G=4.0):
        w = synth.droplet(n=32, r=6.0, seed=4, prec=prec, salt=1e-3, Ez=Ez_, charge=Q_, steps=nsteps, G=G)
        w.params.poisson_tol = 1e-12
        w.params.poisson_max_iter = 500
        return w

    dn = make(Ez, 1.0).n - make(Ez, 0.0).n
    s = gpu_for(make(Ez, Q), lbeh)
    g = s.step_adjoint(nsteps, 10, d_deformation=1.0, dn0_dQ=dn)
    s.close()
    assert g["status"] == lbeh.LBEH_OK

    def oracle_D(w):
        o = oracle_for(w)
        for _ in range(nsteps):
            o.step()
        return observables.deformation(o.densities())[0]

    # central differences with relative step 1e-4: larger steps pick up the
    # non-smooth terms of the step (upwind |u|, the max(0, c) weight of D)
    h = Ez * 1e-4
    fd_E = (oracle_D(make(Ez + h, Q)) - oracle_D(make(Ez - h, Q))) / (2 * h)
    assert abs(g["dE_ext"][2] - fd_E) <= 1e-4 * abs(fd_E), (g["dE_ext"][2], fd_E)
    # Shan-Chen coupling G: the oracle's central differences carry a
    # first-order error from the non-smooth terms (measured 1.3e-4 relative at
    # step 1e-4 of G, falling in proportion to the step), so the adjoint is
    # compared with their extrapolation to zero step, 2 d(h) - d(2h) at
    # relative steps 2.5e-5 and 5e-5 (measured agreement 3e-6)
    fd_G = []
    for rel in (2.5e-5, 5e-5):
        hG = 4.0 * rel
        fd_G.append((oracle_D(make(Ez, Q, G=4.0 + hG)) - oracle_D(make(Ez, Q, G=4.0 - hG))) / (2 * hG))
    fd_G0 = 2.0 * fd_G[0] - fd_G[1]
    assert abs(g["dG"] - fd_G0) <= 1e-4 * abs(fd_G0), (g["dG"], fd_G)
    # dD/dQ is about 1e-5 of dD/dE_z here, so its differences sit near the
    # noise of the two Poisson solves: the noise is the spread of the
    # estimates over three step sizes and the agreement required is
    # max(1e-4, 3 x spread) relative to the central estimate
    fd_Q = []
    for rel in (5e-5, 1e-4, 2e-4):
        hq = Q * rel
        fd_Q.append((oracle_D(make(Ez, Q + hq)) - oracle_D(make(Ez, Q - hq))) / (2 * hq))
    noise = max(fd_Q) - min(fd_Q)
    assert abs(g["dQ"] - fd_Q[1]) <= max(1e-4 * abs(fd_Q[1]), 3.0 * noise), (g["dQ"], fd_Q)

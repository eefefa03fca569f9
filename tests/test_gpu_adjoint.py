"""Discrete adjoint of the coupled step (lbeh_step_adjoint).

Checks, all in FP64 unless stated: a one-step dot-product test of the whole
adjoint step against central differences of the forward step with random
seeds and directions; parameter gradients of the drop deformation after
several steps (E_z, G, drop charge Q) against central finite differences of
the GPU forward and of the oracle; independence from the checkpoint
interval; the FP32 adjoint against the FP64 adjoint."""
import numpy as np
import pytest

import synth
from _common import load, oracle_for

pytestmark = pytest.mark.gpu


def _drop(n=16, prec="fp64", Ez=2e-2, Q=5.0, G=4.0, tol=1e-13, nions=2):
    w = synth.droplet(n=n, r=0.3 * n, seed=5, prec=prec, salt=1e-3, Ez=Ez, charge=Q, steps=1, nions=nions)
    w.params.G = G
    w.params.poisson_tol = tol
    w.params.poisson_max_iter = 500
    return w


def _sys(lbeh, w):
    return load(lbeh.System(w.params), w)


def _deformation_after(lbeh, w, nsteps):
    s = _sys(lbeh, w)
    assert s.step(nsteps) == lbeh.LBEH_OK
    d = s.observables().deformation
    s.close()
    return d


@pytest.mark.parametrize("nions", [2, 0])
def test_one_step_dot_product(lbeh, nions):
    """<adjoint(x_bar), dx> = d/dh <x_bar, step(x + h dx)> for random seeds and
    directions.  A uniform background flow keeps every velocity component far
    from zero, where the upwind advection flux |u| n has its kink and central
    differences would not follow the derivative."""
    w = _drop(nions=nions)
    w.u = np.empty((3,) + w.rho.shape[1:])
    w.u[0], w.u[1], w.u[2] = 0.04, -0.03, 0.05
    s = _sys(lbeh, w)
    assert s.step(3) == lbeh.LBEH_OK  # develop a flow and ion fluxes
    st = s.get(("rho", "n"), f=True)
    f0 = st["f"]
    n0 = st["n"] if nions else None
    s.close()
    rng = np.random.default_rng(11)
    fbar = rng.uniform(-1, 1, size=f0.shape)
    nbar = rng.uniform(-1, 1, size=n0.shape) if nions else None
    df = rng.uniform(-1, 1, size=f0.shape) * 1e-2
    dn = rng.uniform(-1, 1, size=n0.shape) * 1e-4 if nions else None

    def run(h):
        t = lbeh.System(w.params)
        t.set_fields(f=f0 + h * df, n=list(n0 + h * dn) if nions else None)
        assert t.step(1) == lbeh.LBEH_OK
        o = t.get(("n",), f=True)
        t.close()
        J = float((fbar * o["f"]).sum())
        if nions:
            J += float((nbar * o["n"]).sum())
        return J

    h = 1e-4
    fd = (run(h) - run(-h)) / (2 * h)
    t = lbeh.System(w.params)
    t.set_fields(f=f0, n=list(n0) if nions else None)
    g = t.step_adjoint(1, 1, d_deformation=0.0, f_bar=fbar, n_bar=nbar, want_state=True)
    t.close()
    assert g["status"] == lbeh.LBEH_OK
    ad = float((g["f0_bar"] * df).sum())
    if nions:
        ad += float((g["n0_bar"] * dn).sum())
    assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)


def _fd(lbeh, make, x0, rel, nsteps):
    h = abs(x0) * rel
    return (_deformation_after(lbeh, make(x0 + h), nsteps) - _deformation_after(lbeh, make(x0 - h), nsteps)) / (2 * h)


def test_parameter_gradients_match_finite_differences(lbeh):
    nsteps, Ez, G, Q = 8, 2e-2, 4.0, 5.0
    w = _drop(Ez=Ez, G=G, Q=Q)
    dn = _drop(Q=1.0).n - _drop(Q=0.0).n  # initial ions are linear in Q
    s = _sys(lbeh, w)
    g = s.step_adjoint(nsteps, 3, d_deformation=1.0, dn0_dQ=dn)
    s.close()
    assert g["status"] == lbeh.LBEH_OK
    assert abs(g["deformation"] - _deformation_after(lbeh, w, nsteps)) < 1e-14
    fd_E = _fd(lbeh, lambda v: _drop(Ez=v, G=G, Q=Q), Ez, 1e-4, nsteps)
    fd_G = _fd(lbeh, lambda v: _drop(Ez=Ez, G=v, Q=Q), G, 1e-4, nsteps)
    fd_Q = _fd(lbeh, lambda v: _drop(Ez=Ez, G=G, Q=v), Q, 1e-4, nsteps)
    assert abs(g["dE_ext"][2] - fd_E) <= 1e-4 * abs(fd_E), (g["dE_ext"][2], fd_E)
    assert abs(g["dG"] - fd_G) <= 1e-4 * abs(fd_G), (g["dG"], fd_G)
    assert abs(g["dQ"] - fd_Q) <= 1e-4 * abs(fd_Q), (g["dQ"], fd_Q)


def test_gradient_matches_oracle_finite_difference(lbeh):
    from oracle import observables
    nsteps, Ez = 6, 2e-2
    w = _drop(Ez=Ez)
    s = _sys(lbeh, w)
    g = s.step_adjoint(nsteps, 2, d_deformation=1.0)
    s.close()

    def oracle_D(v):
        o = oracle_for(_drop(Ez=v, tol=1e-12))
        for _ in range(nsteps):
            o.step()
        return observables.deformation(o.densities())[0]

    h = Ez * 1e-4
    fd = (oracle_D(Ez + h) - oracle_D(Ez - h)) / (2 * h)
    assert abs(g["dE_ext"][2] - fd) <= 1e-4 * abs(fd), (g["dE_ext"][2], fd)


def test_checkpoint_interval_does_not_change_the_gradient(lbeh):
    w = _drop()
    res = []
    for K in (1, 4, 9):
        s = _sys(lbeh, w)
        g = s.step_adjoint(9, K, d_deformation=1.0, want_state=True)
        s.close()
        res.append(g)
    for g in res[1:]:
        assert np.array_equal(g["dE_ext"], res[0]["dE_ext"]) and g["dG"] == res[0]["dG"]
        assert np.array_equal(g["f0_bar"], res[0]["f0_bar"])


def test_fp32_adjoint_close_to_fp64(lbeh):
    nsteps = 10
    g = {}
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-7)):
        w = _drop(n=24, prec=prec, tol=tol)
        s = _sys(lbeh, w)
        g[prec] = s.step_adjoint(nsteps, 5, d_deformation=1.0)
        s.close()
    assert abs(g["fp32"]["dE_ext"][2] - g["fp64"]["dE_ext"][2]) <= 1e-3 * abs(g["fp64"]["dE_ext"][2])
    assert abs(g["fp32"]["dG"] - g["fp64"]["dG"]) <= 1e-2 * abs(g["fp64"]["dG"])


def test_autograd_function_returns_the_adjoint_gradients(lbeh):
    torch = pytest.importorskip("torch")
    from paper_1712_08494_gb300.autograd import deformation
    nsteps = 5
    dn = _drop(Q=1.0).n - _drop(Q=0.0).n

    def factory(E, G, Q):
        w = _drop(Ez=E[2], G=G, Q=Q)
        return _sys(lbeh, w)

    E = torch.tensor([0.0, 0.0, 2e-2], dtype=torch.float64, requires_grad=True)
    G = torch.tensor(4.0, dtype=torch.float64, requires_grad=True)
    Q = torch.tensor(5.0, dtype=torch.float64, requires_grad=True)
    D = deformation(factory, E, G, Q, nsteps, 2, dn)
    (3.0 * D).backward()
    s = factory([0.0, 0.0, 2e-2], 4.0, 5.0)
    g = s.step_adjoint(nsteps, 2, d_deformation=1.0, dn0_dQ=dn)
    s.close()
    assert float(D.detach()) == g["deformation"]
    assert np.allclose(E.grad.numpy(), 3.0 * g["dE_ext"], rtol=0, atol=0)
    assert float(G.grad) == 3.0 * g["dG"] and float(Q.grad) == 3.0 * g["dQ"]

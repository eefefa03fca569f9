"""Shared helpers of the parity tests: run the same seeded workload through the
CUDA library (C-ABI via the binding) and through the CPU oracle."""
import copy

import numpy as np

from oracle import OracleSystem


def oracle_for(w, phi=None):
    return OracleSystem(w.params, w.rho, w.n, w.u, w.colloid_x if len(w.colloid_r) else None,
                        w.colloid_v if len(w.colloid_r) else None,
                        w.colloid_q if len(w.colloid_r) else None,
                        w.colloid_r if len(w.colloid_r) else None, phi)


def gpu_for(w, lbeh, stream=0):
    return load(lbeh.System(w.params, stream), w)


def load(s, w):
    """Load workload w into the System (or box view) s."""
    nc = len(w.colloid_r)
    s.set_fields(rho=list(w.rho), n=list(w.n) if w.n is not None else None, u=w.u,
                 colloid_x=w.colloid_x if nc else None, colloid_v=w.colloid_v if nc else None,
                 colloid_q=w.colloid_q if nc else None, colloid_r=w.colloid_r if nc else None)
    return s


def step_both(sg, so, nsteps, lbeh=None):
    """Advance both sides; every Poisson solve must reach its tolerance."""
    for _ in range(nsteps):
        so.step()
        rc = sg.step(1)
        assert rc == 0, "lbeh_step status %d" % rc
        if so.nions or so.qc.any() or any(so.E_ext):
            assert so.poisson_relres < so.tol, (so.poisson_relres, so.tol)


def rel_err(a, b):
    """max |a - b| / max |b| (0 when both vanish)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    num = np.abs(a - b).max()
    if den == 0:
        return float(num)
    return float(num / den)


def compare(sg, so, fields=("rho", "n", "phi", "u")):
    got = sg.get(fields)
    errs = {}
    if "rho" in fields:
        errs["rho"] = max(rel_err(got["rho"][s], so.densities()[s]) for s in range(so.ncomp))
    if "n" in fields and so.nions:
        errs["n"] = max(rel_err(got["n"][s], so.n[s]) for s in range(2))
    if "phi" in fields:
        errs["phi"] = rel_err(got["phi"], so.phi)
    if "u" in fields and hasattr(so, "last_u"):
        errs["u"] = rel_err(got["u"], so.last_u)
    return errs


def with_params(w, **kw):
    w = copy.deepcopy(w)
    for k, v in kw.items():
        setattr(w.params, k, v)
    return w

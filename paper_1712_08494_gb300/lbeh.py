"""Python binding of the lbeh C-ABI (include/lbeh.h): argument marshalling only.

Every step of the coupled lattice timestep runs in the CUDA library
``_lib/liblbeh.so``; this module only fills the C structs, passes pointers
(numpy host buffers or torch CUDA tensors) and checks status codes.  There is
no CPU fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbeh.so")

LBEH_OK = 0
LBEH_ERR_INVALID_ARG = -1
LBEH_ERR_OOM = -2
LBEH_ERR_CUDA = -3
LBEH_ERR_POISSON_NOT_CONVERGED = -4
LBEH_ERR_NONFINITE = -5
LBEH_ERR_BARRIER_TIMEOUT = -6
LBEH_ERR_UNSUPPORTED = -7

LBEH_FP64, LBEH_FP32, LBEH_FP32_BF16STORE, LBEH_FP32_FP16STORE = 0, 1, 2, 3
PREC = {"fp64": LBEH_FP64, "fp32": LBEH_FP32, "bf16": LBEH_FP32_BF16STORE, "fp16": LBEH_FP32_FP16STORE}
LBEH_F64, LBEH_F32 = 0, 1
LBEH_POISSON_AUTO, LBEH_POISSON_MULTIGRID, LBEH_POISSON_SPECTRAL = 0, 1, 2
SOLVER = {"auto": LBEH_POISSON_AUTO, "multigrid": LBEH_POISSON_MULTIGRID, "spectral": LBEH_POISSON_SPECTRAL}

LBEH_AUX_SOLID, LBEH_AUX_OWNER, LBEH_AUX_PSI_S, LBEH_AUX_SURFACE = 0, 1, 2, 3
LBEH_AUX_QC, LBEH_AUX_EPS, LBEH_AUX_Q, LBEH_AUX_RHO_V, LBEH_AUX_U = 4, 5, 6, 7, 8

# exported symbols declared in include/lbeh.h
SYMBOLS = ("lbeh_create", "lbeh_set_fields", "lbeh_get_fields", "lbeh_step", "lbeh_observables",
           "lbeh_get_aux", "lbeh_profile_enable", "lbeh_profile_read", "lbeh_observables_noalloc",
           "lbeh_last_error", "lbeh_destroy", "lbeh_status_string", "lbeh_set_wait_limit")
LBEH_NOALLOC_MAX_SITES = 16777216

LBEH_STAGE_MACRO, LBEH_STAGE_POISSON, LBEH_STAGE_COLLIDE, LBEH_STAGE_NP, LBEH_STAGE_COLLOID = 0, 1, 2, 3, 4
LBEH_NSTAGES = 5
STAGE_NAMES = ("macro", "poisson", "collide", "np", "colloid")


class lbeh_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("ncomp", C.c_int), ("nions", C.c_int), ("prec", C.c_int),
        ("tau", C.c_double), ("G", C.c_double), ("rho0_shift", C.c_double * 2),
        ("D", C.c_double), ("bjerrum", C.c_double), ("eps_r", C.c_double * 2),
        ("eps_r_colloid", C.c_double), ("dmu", C.c_double * 2), ("drho_a", C.c_double),
        ("E_ext", C.c_double * 3), ("poisson_tol", C.c_double), ("poisson_max_iter", C.c_int),
        ("ncolloid_max", C.c_int), ("rho_p", C.c_double), ("k_hertz", C.c_double),
        ("psi_subdiv", C.c_int), ("colloids_move", C.c_int), ("stream", C.c_void_p),
        ("poisson_solver", C.c_int),
    ]


class lbeh_fields(C.Structure):
    _fields_ = [
        ("dtype", C.c_int), ("on_device", C.c_int),
        ("rho", C.c_void_p * 2), ("u", C.c_void_p), ("f", C.c_void_p),
        ("n", C.c_void_p * 2), ("phi", C.c_void_p),
        ("ncolloid", C.c_int),
        ("cx", C.POINTER(C.c_double)), ("cv", C.POINTER(C.c_double)),
        ("cq", C.POINTER(C.c_double)), ("cr", C.POINTER(C.c_double)),
        ("cf", C.POINTER(C.c_double)),
    ]


class lbeh_obs(C.Structure):
    _fields_ = [
        ("mass", C.c_double * 2), ("ions", C.c_double * 2), ("charge", C.c_double),
        ("momentum", C.c_double * 3), ("deformation", C.c_double), ("centroid", C.c_double * 3),
        ("colloid_v", C.c_double * 3), ("poisson_relres", C.c_double), ("poisson_iters", C.c_int),
        ("status", C.c_int), ("steps", C.c_longlong), ("poisson_solver", C.c_int),
    ]


class lbeh_obs_seed(C.Structure):
    _fields_ = [("d_deformation", C.c_double), ("f_bar", C.c_void_p), ("n_bar", C.c_void_p),
                ("on_device", C.c_int)]


class lbeh_grads(C.Structure):
    _fields_ = [("deformation", C.c_double), ("dE_ext", C.c_double * 3), ("dG", C.c_double), ("dQ", C.c_double),
                ("dn0_dQ", C.c_void_p), ("f0_bar", C.c_void_p), ("n0_bar", C.c_void_p), ("on_device", C.c_int),
                ("forward_ms", C.c_double), ("adjoint_ms", C.c_double), ("adjoint_poisson_cycles", C.c_longlong)]


class lbeh_profile(C.Structure):
    _fields_ = [("ms", C.c_double * LBEH_NSTAGES), ("calls", C.c_longlong * LBEH_NSTAGES),
                ("launches", C.c_longlong), ("poisson_cycles", C.c_longlong)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbeh.so is not built (%s); run paper_1712_08494_gb300.build()" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    H = C.c_void_p
    lib.lbeh_create.argtypes = [C.POINTER(lbeh_params), C.POINTER(H)]
    lib.lbeh_set_fields.argtypes = [H, C.POINTER(lbeh_fields)]
    lib.lbeh_get_fields.argtypes = [H, C.POINTER(lbeh_fields)]
    lib.lbeh_step.argtypes = [H, C.c_int]
    lib.lbeh_observables.argtypes = [H, C.POINTER(lbeh_obs)]
    lib.lbeh_get_aux.argtypes = [H, C.c_int, C.c_void_p]
    lib.lbeh_profile_enable.argtypes = [H, C.c_int]
    lib.lbeh_profile_read.argtypes = [H, C.POINTER(lbeh_profile)]
    lib.lbeh_observables_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(lbeh_obs), C.c_void_p]
    lib.lbeh_create_batch.argtypes = [C.POINTER(lbeh_params), C.c_int, C.POINTER(H)]
    lib.lbeh_batch_box.argtypes = [H, C.c_int, C.POINTER(H)]
    lib.lbeh_batch_step_sequential.argtypes = [H, C.c_int]
    lib.lbeh_batch_tune.argtypes = [H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.lbeh_batch_set_shape.argtypes = [H, C.c_int]
    lib.lbeh_batch_shape.argtypes = [H]
    lib.lbeh_step_adjoint.argtypes = [H, C.c_int, C.c_int, C.POINTER(lbeh_obs_seed), C.POINTER(lbeh_grads)]
    lib.lbeh_set_wait_limit.argtypes = [H, C.c_longlong]
    lib.lbeh_destroy.argtypes = [H]
    lib.lbeh_destroy.restype = None
    lib.lbeh_last_error.argtypes = [H]
    lib.lbeh_last_error.restype = C.c_char_p
    lib.lbeh_status_string.argtypes = [C.c_int]
    lib.lbeh_status_string.restype = C.c_char_p
    for name in ("lbeh_create", "lbeh_set_fields", "lbeh_get_fields", "lbeh_step", "lbeh_observables",
                 "lbeh_get_aux", "lbeh_profile_enable", "lbeh_profile_read", "lbeh_observables_noalloc",
                 "lbeh_create_batch", "lbeh_batch_box", "lbeh_batch_step_sequential", "lbeh_batch_tune",
                 "lbeh_batch_set_shape", "lbeh_batch_shape", "lbeh_step_adjoint"):
        getattr(lib, name).restype = C.c_int
    return lib


_lib = _load()


class LbehError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, lbeh_status_string(code), code))


def _check(code: int, where: str) -> int:
    if code != LBEH_OK:
        raise LbehError(code, where)
    return code


# ------------------------------------------------------------ raw C-ABI names
def lbeh_status_string(code: int) -> str:
    return _lib.lbeh_status_string(int(code)).decode()


def lbeh_create(params: lbeh_params) -> C.c_void_p:
    h = C.c_void_p()
    _check(_lib.lbeh_create(C.byref(params), C.byref(h)), "lbeh_create")
    return h


def lbeh_set_fields(h, fields: lbeh_fields) -> int:
    return _check(_lib.lbeh_set_fields(h, C.byref(fields)), "lbeh_set_fields")


def lbeh_get_fields(h, fields: lbeh_fields) -> int:
    return _check(_lib.lbeh_get_fields(h, C.byref(fields)), "lbeh_get_fields")


def lbeh_last_error(h) -> str:
    return _lib.lbeh_last_error(h).decode()


def lbeh_step(h, nsteps: int) -> int:
    """Returns the status code; raises only on hard errors (not on a Poisson
    solve that missed its tolerance, which is reported by the status)."""
    rc = _lib.lbeh_step(h, int(nsteps))
    if rc not in (LBEH_OK, LBEH_ERR_POISSON_NOT_CONVERGED):
        raise LbehError(rc, "lbeh_step [%s]" % lbeh_last_error(h))
    return rc


def lbeh_observables(h) -> lbeh_obs:
    o = lbeh_obs()
    _check(_lib.lbeh_observables(h, C.byref(o)), "lbeh_observables")
    return o


def lbeh_get_aux(h, which: int, out: np.ndarray) -> np.ndarray:
    assert out.flags.c_contiguous
    _check(_lib.lbeh_get_aux(h, int(which), out.ctypes.data_as(C.c_void_p)), "lbeh_get_aux")
    return out


def lbeh_profile_enable(h, on: bool = True) -> int:
    return _check(_lib.lbeh_profile_enable(h, 1 if on else 0), "lbeh_profile_enable")


def lbeh_profile_read(h) -> lbeh_profile:
    p = lbeh_profile()
    _check(_lib.lbeh_profile_read(h, C.byref(p)), "lbeh_profile_read")
    return p


def lbeh_observables_noalloc(nx, ny, nz, ncomp, nions, dtype, f_ptr, n_ptr=None, solid_ptr=None, qc_ptr=None,
                             stream=0) -> lbeh_obs:
    """Allocation-free observables over caller-owned device buffers (pointers
    as integers); for callers that cannot allocate device memory."""
    o = lbeh_obs()
    _check(_lib.lbeh_observables_noalloc(int(nx), int(ny), int(nz), int(ncomp), int(nions), int(dtype), f_ptr,
                                         n_ptr, solid_ptr, qc_ptr, C.byref(o), int(stream) or None),
           "lbeh_observables_noalloc")
    return o


def lbeh_step_adjoint(h, nsteps: int, ckpt_every: int, seed: lbeh_obs_seed, grads: lbeh_grads) -> int:
    rc = _lib.lbeh_step_adjoint(h, int(nsteps), int(ckpt_every), C.byref(seed), C.byref(grads))
    if rc not in (LBEH_OK, LBEH_ERR_POISSON_NOT_CONVERGED):
        raise LbehError(rc, "lbeh_step_adjoint [%s]" % lbeh_last_error(h))
    return rc


def lbeh_create_batch(params_list) -> C.c_void_p:
    arr = (lbeh_params * len(params_list))(*params_list)
    h = C.c_void_p()
    _check(_lib.lbeh_create_batch(arr, len(params_list), C.byref(h)), "lbeh_create_batch")
    return h


def lbeh_batch_box(h, b: int) -> C.c_void_p:
    box = C.c_void_p()
    _check(_lib.lbeh_batch_box(h, int(b), C.byref(box)), "lbeh_batch_box")
    return box


def lbeh_batch_step_sequential(h, nsteps: int) -> int:
    rc = _lib.lbeh_batch_step_sequential(h, int(nsteps))
    if rc not in (LBEH_OK, LBEH_ERR_POISSON_NOT_CONVERGED):
        raise LbehError(rc, "lbeh_batch_step_sequential [%s]" % lbeh_last_error(h))
    return rc


def lbeh_batch_tune(h, probe_steps: int):
    cpb = C.c_int()
    ms = C.c_double()
    _check(_lib.lbeh_batch_tune(h, int(probe_steps), C.byref(cpb), C.byref(ms)), "lbeh_batch_tune")
    return cpb.value, ms.value


def lbeh_batch_set_shape(h, cluster_blocks: int) -> int:
    return _check(_lib.lbeh_batch_set_shape(h, int(cluster_blocks)), "lbeh_batch_set_shape")


def lbeh_batch_shape(h) -> int:
    return int(_lib.lbeh_batch_shape(h))


def lbeh_set_wait_limit(h, polls: int) -> int:
    return _check(_lib.lbeh_set_wait_limit(h, int(polls)), "lbeh_set_wait_limit")


def lbeh_destroy(h) -> None:
    _lib.lbeh_destroy(h)


# ------------------------------------------------------------ marshalling helpers
def make_params(p, stream: int = 0) -> lbeh_params:
    """Fill lbeh_params from any object with the attributes of synth.Params."""
    c = lbeh_params()
    c.nx, c.ny, c.nz = int(p.nx), int(p.ny), int(p.nz)
    c.ncomp, c.nions = int(p.ncomp), int(p.nions)
    c.prec = PREC[p.prec] if isinstance(p.prec, str) else int(p.prec)
    c.tau, c.G = float(p.tau), float(p.G)
    c.rho0_shift[0], c.rho0_shift[1] = float(p.rho0_shift[0]), float(p.rho0_shift[1])
    c.D, c.bjerrum = float(p.D), float(p.bjerrum)
    c.eps_r[0], c.eps_r[1] = float(p.eps_r[0]), float(p.eps_r[1])
    c.eps_r_colloid = float(p.eps_r_colloid)
    c.dmu[0], c.dmu[1] = float(p.dmu[0]), float(p.dmu[1])
    c.drho_a = float(p.drho_a)
    for a in range(3):
        c.E_ext[a] = float(p.E_ext[a])
    c.poisson_tol, c.poisson_max_iter = float(p.poisson_tol), int(p.poisson_max_iter)
    c.ncolloid_max = int(p.ncolloid_max)
    c.rho_p, c.k_hertz = float(p.rho_p), float(p.k_hertz)
    c.psi_subdiv, c.colloids_move = int(p.psi_subdiv), int(p.colloids_move)
    c.stream = int(stream) or None
    sv = getattr(p, "poisson_solver", "auto")
    c.poisson_solver = SOLVER[sv] if isinstance(sv, str) else int(sv)
    return c


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    return int(a.data_ptr())  # torch tensor


def _dptr(a):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


class System:
    """One lattice system behind an lbeh handle (marshalling only).

    Field arguments are numpy arrays (host) or torch CUDA tensors (device) of
    float64 or float32, shaped like the C-ABI layout."""

    def __init__(self, params, stream: int = 0, handle=None):
        self.params = params
        self.cparams = make_params(params, stream)
        # handle: a box of a batch (owned by the batch, not released here)
        self.owned = handle is None
        self.h = lbeh_create(self.cparams) if handle is None else handle
        self.N = int(params.nx) * int(params.ny) * int(params.nz)
        self.shape = (int(params.nz), int(params.ny), int(params.nx))
        self.ncomp = int(params.ncomp)
        self.nions = int(params.nions)
        self._keep = []

    def close(self):
        if self.h:
            if self.owned:
                lbeh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _kind(arrs):
        for a in arrs:
            if a is None:
                continue
            if isinstance(a, np.ndarray):
                return (LBEH_F64 if a.dtype == np.float64 else LBEH_F32), 0
            import torch
            return (LBEH_F64 if a.dtype == torch.float64 else LBEH_F32), (1 if a.is_cuda else 0)
        return LBEH_F64, 0

    def set_fields(self, rho=None, n=None, u=None, f=None, phi=None, colloid_x=None, colloid_v=None,
                   colloid_q=None, colloid_r=None):
        fl = lbeh_fields()
        rho_list = list(rho) if rho is not None else [None, None]
        n_list = list(n) if n is not None else [None, None]
        arrs = rho_list + n_list + [u, f, phi]
        fl.dtype, fl.on_device = self._kind(arrs)
        keep = []

        def conv(a):
            if a is None:
                return None
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=np.float64 if fl.dtype == LBEH_F64 else np.float32)
            else:
                a = a.contiguous()
            keep.append(a)
            return _ptr(a)

        for s in range(min(2, len(rho_list))):
            fl.rho[s] = conv(rho_list[s])
        for s in range(min(2, len(n_list))):
            fl.n[s] = conv(n_list[s])
        fl.u = conv(u)
        fl.f = conv(f)
        fl.phi = conv(phi)
        nc = 0 if colloid_x is None else int(np.asarray(colloid_x).reshape(-1, 3).shape[0])
        fl.ncolloid = nc
        if nc:
            for name, arr in (("cx", colloid_x), ("cv", colloid_v), ("cq", colloid_q), ("cr", colloid_r)):
                if arr is None:
                    continue
                a, p = _dptr(arr)
                keep.append(a)
                setattr(fl, name, p)
        lbeh_set_fields(self.h, fl)
        self._keep = keep

    def step(self, nsteps: int = 1) -> int:
        return lbeh_step(self.h, nsteps)

    def observables(self) -> lbeh_obs:
        return lbeh_observables(self.h)

    def step_adjoint(self, nsteps: int, ckpt_every: int, d_deformation: float = 1.0, f_bar=None, n_bar=None,
                     dn0_dQ=None, want_state: bool = False) -> dict:
        """Advance nsteps and return the gradients of the objective (host FP64
        arrays in, host FP64 arrays out)."""
        keep = []

        def host(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data

        seed = lbeh_obs_seed()
        seed.d_deformation = float(d_deformation)
        seed.f_bar = host(f_bar)
        seed.n_bar = host(n_bar)
        seed.on_device = 0
        g = lbeh_grads()
        g.dn0_dQ = host(dn0_dQ)
        g.on_device = 0
        out = {}
        if want_state:
            out["f0_bar"] = np.zeros((self.ncomp, 19) + self.shape)
            g.f0_bar = out["f0_bar"].ctypes.data
            out["n0_bar"] = np.zeros((2,) + self.shape)
            g.n0_bar = out["n0_bar"].ctypes.data
        out["status"] = lbeh_step_adjoint(self.h, nsteps, ckpt_every, seed, g)
        out.update(deformation=g.deformation, dE_ext=np.array(g.dE_ext[:]), dG=g.dG, dQ=g.dQ,
                   forward_ms=g.forward_ms, adjoint_ms=g.adjoint_ms, adjoint_poisson_cycles=g.adjoint_poisson_cycles)
        return out

    def profile_enable(self, on: bool = True):
        lbeh_profile_enable(self.h, on)

    def profile_read(self) -> dict:
        p = lbeh_profile_read(self.h)
        return {"ms": {STAGE_NAMES[k]: p.ms[k] for k in range(LBEH_NSTAGES)},
                "calls": {STAGE_NAMES[k]: p.calls[k] for k in range(LBEH_NSTAGES)},
                "launches": p.launches, "poisson_cycles": p.poisson_cycles}

    def get(self, what=("rho", "n", "phi", "u"), f=False):
        """Host FP64 copies of the requested fields."""
        fl = lbeh_fields()
        fl.dtype, fl.on_device = LBEH_F64, 0
        out = {}
        if "rho" in what:
            out["rho"] = np.zeros((self.ncomp,) + self.shape)
            for s in range(self.ncomp):
                fl.rho[s] = out["rho"][s].ctypes.data
        if "n" in what and self.nions:
            out["n"] = np.zeros((2,) + self.shape)
            for s in range(2):
                fl.n[s] = out["n"][s].ctypes.data
        if "phi" in what:
            out["phi"] = np.zeros(self.shape)
            fl.phi = out["phi"].ctypes.data
        if "u" in what:
            out["u"] = np.zeros((3,) + self.shape)
            fl.u = out["u"].ctypes.data
        if f:
            out["f"] = np.zeros((self.ncomp, 19) + self.shape)
            fl.f = out["f"].ctypes.data
        ncmax = int(self.params.ncolloid_max)
        if ncmax:
            for name in ("cx", "cv", "cf"):
                arr = np.zeros((ncmax, 3))
                out[name] = arr
                setattr(fl, name, arr.ctypes.data_as(C.POINTER(C.c_double)))
        lbeh_get_fields(self.h, fl)
        if ncmax:
            for name in ("cx", "cv", "cf"):
                out[name] = out[name][:fl.ncolloid]
        return out

    def aux(self, which: int):
        shp = self.shape
        if which in (LBEH_AUX_SOLID, LBEH_AUX_SURFACE):
            out = np.zeros(shp, dtype=np.uint8)
        elif which == LBEH_AUX_OWNER:
            out = np.zeros(shp, dtype=np.int32)
        elif which == LBEH_AUX_RHO_V:
            out = np.zeros((self.ncomp,) + shp)
        elif which == LBEH_AUX_U:
            out = np.zeros((3,) + shp)
        else:
            out = np.zeros(shp)
        return lbeh_get_aux(self.h, which, out)


class Batch:
    """Independent systems advanced together by one launch per step call
    (marshalling only); box b is a System view owned by the batch."""

    def __init__(self, params_list, stream: int = 0):
        self.params = list(params_list)
        self.h = lbeh_create_batch([make_params(p, stream) for p in self.params])
        self.boxes = [System(p, stream, handle=lbeh_batch_box(self.h, b)) for b, p in enumerate(self.params)]

    def step(self, nsteps: int = 1) -> int:
        return lbeh_step(self.h, nsteps)

    def step_sequential(self, nsteps: int = 1) -> int:
        return lbeh_batch_step_sequential(self.h, nsteps)

    def tune(self, probe_steps: int = 4):
        return lbeh_batch_tune(self.h, probe_steps)

    def set_shape(self, cluster_blocks: int):
        lbeh_batch_set_shape(self.h, cluster_blocks)

    def shape(self) -> int:
        return lbeh_batch_shape(self.h)

    def close(self):
        if self.h:
            for b in self.boxes:
                b.h = None
            lbeh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Allocation-free observables entry point (lbeh_observables_noalloc).

This variant serves callers that cannot allocate device memory where they
need the conserved sums (code under a fixed memory budget, plugins holding
only borrowed device buffers, processes whose allocator belongs to another
runtime).  It keeps
its partial sums in a static device array instead of handle-owned scratch.
The test feeds it the device copies of a system's fields and checks, on two
calls in a row, that it reports what lbeh_observables reports for the same
state, to the FP64 round-off of a different summation order (1e-12 relative).
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from _common import gpu_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbeh():
    import paper_1712_08494_gb300 as pkg
    pkg.build()
    return pkg.load()


def _device_fields(sg, lbeh, torch, dtype):
    """Device copies of the populations and ions written by lbeh_get_fields."""
    tdt = torch.float64 if dtype == lbeh.LBEH_F64 else torch.float32
    f = torch.empty((sg.ncomp, 19) + sg.shape, dtype=tdt, device="cuda")
    n = torch.empty((2,) + sg.shape, dtype=tdt, device="cuda") if sg.nions else None
    fl = lbeh.lbeh_fields()
    fl.dtype, fl.on_device = dtype, 1
    fl.f = f.data_ptr()
    if n is not None:
        fl.n[0] = n[0].data_ptr()
        fl.n[1] = n[1].data_ptr()
    lbeh.lbeh_get_fields(sg.h, fl)
    return f, n


def _close(a, b, scale, tol=1e-12):
    return abs(a - b) <= tol * max(abs(b), scale)


@pytest.mark.parametrize("case", ["droplet_fp32", "slab_colloid_fp64"])
def test_noalloc_observables_match_handle_observables(lbeh, case):
    import torch
    if case == "droplet_fp32":
        w = synth.droplet(n=24, r=7.0, prec="fp32", tol=1e-8, Ez=0.02, charge=4.0)
        dtype = lbeh.LBEH_F32
    else:
        w = synth.two_slab(nx=20, ny=24, nz=28, G=4.0, prec="fp64", tol=1e-12)
        w.colloid_x[:] = [[10.0, 12.0, 13.5]]
        dtype = lbeh.LBEH_F64
    stream = torch.cuda.current_stream()
    sg = gpu_for(w, lbeh, stream.cuda_stream)
    sg.step(3)
    ref = sg.observables()
    f, n = _device_fields(sg, lbeh, torch, dtype)
    solid = qc = None
    if len(w.colloid_r):
        solid = torch.from_numpy(sg.aux(lbeh.LBEH_AUX_SOLID)).cuda()
        qc = torch.from_numpy(sg.aux(lbeh.LBEH_AUX_QC)).cuda()
    torch.cuda.synchronize()
    p = w.params
    mass_scale = sum(ref.mass)
    ion_scale = sum(ref.ions)
    for call in range(2):
        o = lbeh.lbeh_observables_noalloc(
            p.nx, p.ny, p.nz, p.ncomp, p.nions, dtype, f.data_ptr(),
            n.data_ptr() if n is not None else None,
            solid.data_ptr() if solid is not None else None,
            qc.data_ptr() if qc is not None else None, stream.cuda_stream)
        assert o.status == lbeh.LBEH_OK
        for s in range(p.ncomp):
            assert _close(o.mass[s], ref.mass[s], mass_scale), (call, "mass", o.mass[s], ref.mass[s])
        for s in range(2):
            assert _close(o.ions[s], ref.ions[s], ion_scale), (call, "ions")
        assert _close(o.charge, ref.charge, ion_scale), (call, "charge", o.charge, ref.charge)
        for a in range(3):
            assert _close(o.momentum[a], ref.momentum[a], mass_scale), (call, "momentum", a)
            assert _close(o.centroid[a], ref.centroid[a], 1.0), (call, "centroid", a)
        assert _close(o.deformation, ref.deformation, 1.0), (call, "deformation")
    sg.close()


def test_noalloc_rejects_boxes_beyond_its_static_scratch(lbeh):
    import torch
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    # the size check happens on the host, before any kernel sees the buffer
    with pytest.raises(lbeh.LbehError) as e:
        lbeh.lbeh_observables_noalloc(512, 256, 256, 1, 0, lbeh.LBEH_F32, buf.data_ptr(), None, None, None, 0)
    assert e.value.code == lbeh.LBEH_ERR_INVALID_ARG

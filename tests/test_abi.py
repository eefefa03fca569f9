"""The C-ABI library loads, exports every function include/lbeh.h declares, and
its struct layouts match the Python binding (no GPU needed)."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbeh.h")


@pytest.fixture(scope="module")
def lib():
    import paper_1712_08494_gb300 as pkg
    pkg.build()
    from paper_1712_08494_gb300 import lbeh
    return lbeh


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbeh_\w+)\s*\(", txt, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lbeh_step" in names and "lbeh_create" in names
    for n in names:
        assert hasattr(lib._lib, n), n
    assert set(names) <= set(lib.SYMBOLS) | set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lbeh_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_header(lib):
    import ctypes as C
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "lbeh.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(lbeh_params), sizeof(lbeh_fields), sizeof(lbeh_obs), sizeof(lbeh_profile));
  printf("%zu %zu %zu %zu %zu\n", offsetof(lbeh_params, E_ext), offsetof(lbeh_params, stream),
         offsetof(lbeh_fields, ncolloid), offsetof(lbeh_obs, steps), offsetof(lbeh_params, poisson_solver));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(v) for v in lines[0].split()]
    offs = [int(v) for v in lines[1].split()]
    assert sizes == [C.sizeof(lib.lbeh_params), C.sizeof(lib.lbeh_fields), C.sizeof(lib.lbeh_obs),
                     C.sizeof(lib.lbeh_profile)]
    assert offs == [lib.lbeh_params.E_ext.offset, lib.lbeh_params.stream.offset,
                    lib.lbeh_fields.ncolloid.offset, lib.lbeh_obs.steps.offset,
                    lib.lbeh_params.poisson_solver.offset]


def test_invalid_parameters_are_rejected_without_a_device(lib):
    import synth
    bad = [dict(nx=1), dict(ncomp=3), dict(nions=1), dict(prec="fp64", tau=0.5), dict(D=0.0),
           dict(poisson_solver=3)]
    for kw in bad:
        p = synth.Params(nx=8, ny=8, nz=8)
        for k, v in kw.items():
            setattr(p, k, v)
        with pytest.raises(lib.LbehError) as e:
            lib.lbeh_create(lib.make_params(p))
        assert e.value.code == lib.LBEH_ERR_INVALID_ARG
    assert lib.lbeh_status_string(lib.LBEH_ERR_POISSON_NOT_CONVERGED).startswith("Poisson")

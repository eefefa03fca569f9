"""GB300-native coupled electrohydrodynamic lattice step (arXiv:1712.08494, Sec. II).

The compute path is the CUDA library ``_lib/liblbeh.so`` (C-ABI in
``include/lbeh.h``); ``lbeh`` is its Python binding.  Build the library with
``paper_1712_08494_gb300.build()``.
"""
from .buildlib import LIB as LIBRARY_PATH, build  # noqa: F401


def load():
    """Import the binding (raises if the CUDA library is not built)."""
    from . import lbeh
    return lbeh

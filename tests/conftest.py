import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU-only physics validation")


def pytest_collection_modifyitems(config, items):
    """GPU tests are skipped (not failed) where no GPU is visible, so that
    ``-m "not gpu"`` and plain collection work on CPU-only machines."""
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device visible")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="module")
def lbeh():
    """The CUDA library's binding (built in-tree on first use)."""
    import paper_1712_08494_gb300 as pkg
    pkg.build()
    from paper_1712_08494_gb300 import lbeh as L
    return L

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300 / sm_103a)")
    config.addinivalue_line("markers", "slow: longer-running physics check")


@pytest.fixture(scope="session")
def lbm():
    """The CUDA library binding (skips when no GPU is present)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_08766_gb300 as pkg
    pkg.load()
    return pkg


@pytest.fixture(scope="session")
def built_library():
    """The compiled library, built here if needed (nvcc only; no GPU): host tests whose
    code path asks the library for sizes (lbm_domain_bytes) load it without a device."""
    import paper_1901_08766_gb300 as pkg
    pkg.build()
    pkg.load()
    return pkg

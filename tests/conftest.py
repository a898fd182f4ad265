import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built liblbm.so")
    config.addinivalue_line(
        "markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def lbm():
    """The CUDA library through its Python binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0707_2437_gb300 import lbm as lbm_mod
    lbm_mod.load()
    return lbm_mod

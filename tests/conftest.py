import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: long-running case")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def darm():
    """The CUDA library's Python binding, initialised on device 0."""
    if not cuda_available():
        pytest.fail("gpu test selected but no CUDA device is visible")
    import paper_2107_05681_gb300 as d
    d.init(0)
    return d

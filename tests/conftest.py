import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libdctgb")


@pytest.fixture(scope="session")
def lib():
    """The loaded C-ABI library (built on demand; no GPU needed to load)."""
    from paper_1306_1373_gb300 import dctgb
    return dctgb.load()


@pytest.fixture(scope="session")
def cuda_ok():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True

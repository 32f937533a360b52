import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU run (still part of the default suite)")


@pytest.fixture(scope="session")
def qlbm_lib():
    """The CUDA library, built in-tree if needed (nvcc cross-compiles without a GPU)."""
    from paper_2211_16933_gb300 import build as B
    B.build()
    from paper_2211_16933_gb300 import qlbm
    return qlbm


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu(qlbm_lib):
    if not _has_gpu():
        pytest.skip("no CUDA device")
    return qlbm_lib

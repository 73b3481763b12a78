import os
import sys

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if REPO not in sys.path:
    sys.path.insert(0, REPO)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and libgxp.so")
    config.addinivalue_line("markers", "slow: full-size parity case")


def _has_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu():
    """The GPU binding; a gpu-marked test on a machine without a GPU fails loudly."""
    if not _has_gpu():
        pytest.fail("this test is marked gpu but no CUDA device is visible")
    from paper_2203_13005_gb300 import gxp
    return gxp

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle physics runs of tens of seconds on the host")


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library, built for sm_103a; a GPU test fails loudly when it is missing."""
    if not cuda_available():
        pytest.fail("gpu-marked test run without a CUDA device")
    from paper_2106_01557_gb300 import lbm
    return lbm.load()

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def cuda_lib():
    """The built C-ABI library, on a machine with a GPU; fails loudly otherwise."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu-marked test collected on a machine without CUDA")
    from paper_1612_06592_gb300 import lp
    return lp

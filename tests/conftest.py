import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running test")


@pytest.fixture(scope="session")
def cuda_lib():
    """The built C-ABI library on a CUDA device; loading fails loudly if it is missing."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("gpu test collected on a machine without CUDA")
    import paper_2602_20226_gb300 as tt

    tt.load()
    return tt

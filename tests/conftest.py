import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def gpu():
    """The CUDA library through its Python binding; fails loudly when absent."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for a gpu-marked test")
    import paper_2502_10783_gb300 as ipp
    ipp.load()
    return ipp

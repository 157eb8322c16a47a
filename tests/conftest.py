import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: slower CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.oracle.build()
    return oracle


@pytest.fixture(scope="session")
def fea():
    """The CUDA library's Python binding; GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_05872_gb300 as fea
    fea.load()
    return fea

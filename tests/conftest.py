import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs through the C ABI)")
    config.addinivalue_line("markers", "slow: full-size cases (minutes)")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def ipm():
    """The CUDA library, built in-tree; GPU tests fail (not skip) if it is missing."""
    import torch

    from paper_2005_12648_gb300 import build_ext

    build_ext.build_library()
    import paper_2005_12648_gb300 as m

    m.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


@pytest.fixture(scope="session")
def dev(ipm):
    import torch

    return torch.device("cuda:0")

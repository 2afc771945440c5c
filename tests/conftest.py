import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libfgk")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def fgk_mod():
    """The libfgk binding, built in-tree; GPU tests fail (not skip) without CUDA."""
    import torch

    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2508_01864_gb300 import build, fgk

    build.build()
    fgk.load()
    return fgk

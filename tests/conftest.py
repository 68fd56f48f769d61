import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the CUDA library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session")
def dv():
    """The CUDA binding, built in-tree; skips only when no GPU is visible."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_14435_gb300 import dvqls
    return dvqls


@pytest.fixture(scope="session")
def ctx(dv):
    import torch
    h = dv.dvqls_create(0, torch.cuda.current_stream().cuda_stream)
    yield h
    dv.dvqls_destroy(h)

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libmf.so")
    config.addinivalue_line("markers", "slow: large workload (full-size instances)")


@pytest.fixture(scope="session")
def built():
    """Builds the generator, the oracle and libmf.so once per session (no-op when up to date)."""
    import __graft_entry__

    __graft_entry__.build()
    return True


@pytest.fixture(scope="session")
def gpu(built):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a -m gpu test ran without a visible CUDA device")
    from paper_1507_01926_gb300 import mf

    return mf

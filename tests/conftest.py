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
def gpu_lib():
    """The built C-ABI library, loaded through the Python binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_10554_gb300 as iqs
    return iqs


# Run last: the allocation-free call's tests, so that a run which stops at its
# first failure has already run every other test.
RUN_LAST = ("test_probabilities_noalloc.py",)


def pytest_collection_modifyitems(session, config, items):
    last = [it for it in items if it.fspath.basename in RUN_LAST]
    if last:
        items[:] = [it for it in items if it.fspath.basename not in RUN_LAST] + last

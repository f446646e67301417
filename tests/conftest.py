import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line(
        "markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def _wants_fullsize(items):
    return any(os.path.basename(str(it.fspath)) == "test_gpu_fullsize.py" for it in items)


def pytest_collection_finish(session):
    """Start the full-size oracle legs (tests/fullsize_oracle.py) as soon as
    the session knows it will run them, so they overlap the other tests."""
    if not _wants_fullsize(session.items):
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except ImportError:
        return
    from tests import fullsize_oracle
    fullsize_oracle.start()


def pytest_sessionfinish(session, exitstatus):
    from tests import fullsize_oracle
    fullsize_oracle.stop()

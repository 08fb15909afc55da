import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")
if GOLDEN not in sys.path:
    sys.path.insert(0, GOLDEN)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU checks")


@pytest.fixture(scope="session")
def lib():
    """The CUDA library through its Python binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_08847_gb300 import muffin
    return muffin


def pytest_collection_finish(session):
    """When the precision tests are selected on a machine with a GPU, start their
    long FP64 oracle runs now (in spawned worker processes, before any CUDA call
    of this process) so that they overlap the other GPU tests."""
    if not any("test_gpu_precision" in item.nodeid for item in session.items):
        return
    import torch
    if not torch.cuda.is_available():
        return
    import oracle_jobs
    oracle_jobs.start()

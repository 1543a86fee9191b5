import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libfkfast.so")


@pytest.fixture(scope="session")
def fk():
    """The CUDA library binding, built in-tree if needed.  GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06451_gb300 import build, fkfast
    build.build()
    fkfast.load()
    return fkfast

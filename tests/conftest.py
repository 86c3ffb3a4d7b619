import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


def pytest_sessionstart(session):
    """Build the decoder library, the input generators and the oracle when missing or older
    than their sources (each step is a no-op otherwise), so no test runs on a stale build."""
    from paper_2605_10433_gb300 import build as B
    from paper_2605_10433_gb300 import inputs
    import oracle
    from oracle import gf4
    B.build()
    inputs.build_lib()
    oracle.build_lib()
    gf4.build_lib()


@pytest.fixture(scope="session")
def has_gpu():
    import torch
    return torch.cuda.is_available()

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libdpmm.so")
    config.addinivalue_line("markers", "slow: long statistical test")


@pytest.fixture(scope="session")
def tiny_dataset():
    from paper_1812_10048_gb300 import synth
    return synth.tiny()

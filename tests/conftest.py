import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libchemora.so")
    config.addinivalue_line("markers", "slow: full-size parity cases (tens of seconds of oracle time)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle

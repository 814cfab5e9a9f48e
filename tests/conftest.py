import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs on the GB300 box)")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(autouse=True)
def _no_oracle_mutation():
    """Every test starts and ends with the oracle's planted-mistake switch off."""
    import oracle
    oracle.set_mutation(0)
    yield
    oracle.set_mutation(0)

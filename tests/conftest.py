"""Shared fixtures.  Tests marked ``gpu`` need a CUDA device; the rest run on CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); runs the CUDA library through its C ABI")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle

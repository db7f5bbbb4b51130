"""Shared pytest configuration.

Tests marked ``gpu`` need a CUDA device and the in-tree CUDA library; every
other test runs on the CPU (the oracle, host-side logic, the C-ABI's symbol
table and argument checks).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle

"""Shared test configuration.

Markers: ``gpu`` tests need a CUDA device and the compiled library; every
other test runs on the CPU (the oracle, host logic, the C-ABI surface).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libsfhad")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    # keep the no-allocation entry-point test file (if any) last, whatever order
    # pytest found the files in
    items.sort(key=lambda it: 1 if os.path.basename(str(it.fspath)).startswith("test_zz_") else 0)

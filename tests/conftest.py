import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libdvm.so")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


def pytest_ignore_collect(collection_path, config):
    """A GPU-only run (-m gpu) does not collect the randomised oracle properties
    (CPU tests that need hypothesis): where hypothesis is not installed their
    module-level skip would otherwise show as a skipped GPU test."""
    if config.getoption("markexpr", "") == "gpu" and collection_path.name == "test_oracle_properties.py":
        return True
    return None

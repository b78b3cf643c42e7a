import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # long-running tests after the quick ones (a failure there cannot hide them
    # under -x); the allocation-free entry point's file stays last of all
    def key(it):
        last = os.path.basename(str(it.fspath)) == "test_zz_no_alloc.py"
        return (2 if last else (1 if it.get_closest_marker("slow") else 0))
    items.sort(key=key)

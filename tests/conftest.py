import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the compiled libsawave.so")


def pytest_collection_modifyitems(config, items):
    # Keep the file-level order pytest discovers, but make sure files named
    # test_zz_* come last even when tests are selected by marker.
    items.sort(key=lambda it: (os.path.basename(str(it.fspath)).startswith("test_zz_"),))

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU-only case")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped automatically on machines without a device only when
    # they are not explicitly selected; `-m gpu` on a GPU machine runs them all.
    pass

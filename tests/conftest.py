import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "run_last: runs after every other collected test (GPU paths whose first "
                                       "GPU run is still ahead), so that under -x a failure there cannot hide "
                                       "the results of the established tests")


def pytest_collection_modifyitems(config, items):
    first = [it for it in items if it.get_closest_marker("run_last") is None]
    last = [it for it in items if it.get_closest_marker("run_last") is not None]
    items[:] = first + last

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
    config.addinivalue_line("markers", "unverified: GPU code that has not run on a GPU yet; skipped unless "
                                       "MFS_RUN_UNVERIFIED=1")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("MFS_RUN_UNVERIFIED") == "1":
        return
    skip = pytest.mark.skip(reason="GPU path not yet run on a GPU (set MFS_RUN_UNVERIFIED=1 to run it)")
    for item in items:
        if "unverified" in item.keywords:
            item.add_marker(skip)

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def pytest_collection_modifyitems(config, items):
    # A GPU test on a machine without a GPU is an error, not a skip: the CUDA path has
    # no fallback.  Deselection is done with -m "not gpu".
    pass


@pytest.fixture(scope="session", autouse=True)
def built_library():
    """The compiled library every test calls, built once per session if a source is newer
    (nothing is recompiled when it is up to date)."""
    from paper_1509_04681_gb300 import build
    build.build()

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


def pytest_collection_modifyitems(config, items):
    # A GPU test on a machine without a GPU is a configuration error, not a skip:
    # the CPU run selects -m "not gpu" explicitly.
    pass


@pytest.fixture(scope="session")
def oracle_impl():
    import oracle

    return oracle.Oracle()

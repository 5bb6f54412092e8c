import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def pytest_collection_modifyitems(config, items):
    # CPU-only hosts: GPU tests are deselected by -m "not gpu"; when they are selected
    # anyway without a device, fail loudly instead of silently passing.
    pass


@pytest.fixture(scope="session")
def gg():
    import graphgen
    graphgen.build()
    return graphgen


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle

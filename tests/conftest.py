import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def geom():
    from paper_2302_08252_gb300 import workloads
    return workloads.calorimeter()


@pytest.fixture(scope="session")
def otables():
    import oracle
    return oracle.build_tables()


@pytest.fixture(scope="session")
def oworld(geom, otables):
    import oracle
    return oracle.World(geom, otables, seed=1)

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def c1():
    import workloads
    return workloads.starfish_c1()


@pytest.fixture(scope="session")
def c1_oracle(c1):
    import oracle
    o = oracle.Oracle(c1)
    o.brute_force_lists()
    return o


@pytest.fixture(scope="session")
def small():
    import workloads
    return workloads.small_grid()


@pytest.fixture(scope="session")
def small_oracle(small):
    import oracle
    o = oracle.Oracle(small)
    o.brute_force_lists()
    return o

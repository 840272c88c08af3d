import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libvsie")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def sphere_loop_shield():
    from paper_2206_12409_gb300 import inputs as I
    return I.problem_sphere_loop_shield()


@pytest.fixture(scope="session")
def hybrid_parts(sphere_loop_shield):
    from oracle import hybrid
    return hybrid.build_parts(sphere_loop_shield)


@pytest.fixture(scope="session")
def dense_reference(sphere_loop_shield):
    from oracle import hybrid
    return hybrid.dense_operator(sphere_loop_shield)

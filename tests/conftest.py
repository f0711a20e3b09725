import functools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU runs")


@functools.lru_cache(maxsize=None)
def small_problem(name, **over):
    from h2gen import make_problem
    return make_problem(name, **over)


def problem(name, **over):
    return small_problem(name, **over)


@pytest.fixture(scope="session")
def cov2d_1k():
    return problem("cov2d", n=1024, leaf=32)

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


_CACHE = {}


def cached_workload(name, **kw):
    from workloads import make_workload
    key = (name, tuple(sorted(kw.items())))
    if key not in _CACHE:
        _CACHE[key] = make_workload(name, **kw)
    return _CACHE[key]


@pytest.fixture(scope="session")
def wl():
    return cached_workload

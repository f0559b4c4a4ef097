import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test taking more than ~30 s")


_CACHE = {}


def cached(key, fn):
    """Session-wide memo for expensive oracle objects (dense P of a mesh)."""
    if key not in _CACHE:
        _CACHE[key] = fn()
    return _CACHE[key]


@pytest.fixture(scope="session")
def bar_mesh():
    import meshgen
    return meshgen.bar()


@pytest.fixture(scope="session")
def bar_dense_P(bar_mesh):
    from oracle import panels
    return cached("barP", lambda: panels.dense_P(panels.Geometry(bar_mesh.xyz, bar_mesh.tri)))


@pytest.fixture(scope="session")
def two_bars_mesh():
    import meshgen
    return meshgen.two_bars()


@pytest.fixture(scope="session")
def two_bars_dense_P(two_bars_mesh):
    from oracle import panels
    return cached("twoP", lambda: panels.dense_P(panels.Geometry(two_bars_mesh.xyz, two_bars_mesh.tri)))

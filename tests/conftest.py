import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


_cache = {}


def _workload(name, **kw):
    from paper_2304_09953_gb300.workload import make_workload
    key = (name, tuple(sorted(kw.items())))
    if key not in _cache:
        _cache[key] = make_workload(name, **kw)
    return _cache[key]


@pytest.fixture(scope="session")
def tiny():
    """1 ligand, N=24, R=4, 6 x 32^3 maps, 64 x 8 starts, S=8, K=4."""
    return _workload("tiny")


@pytest.fixture(scope="session")
def batched_small():
    """First 64 ligands of the 10k-ligand batched library (same pocket)."""
    return _workload("batched", n_ligands=64)


@pytest.fixture(scope="session")
def workload_factory():
    return _workload

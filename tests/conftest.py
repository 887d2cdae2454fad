"""Shared fixtures.  Tests marked ``gpu`` need a GB300 and the CUDA library;
everything else runs on the CPU (oracle pins, host logic, ABI exports)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


_CACHE = {}


@pytest.fixture(scope="session")
def cfg():
    """cfg(i, walk_num=None) -> cached synthetic workload i."""
    from paper_2512_16677_gb300 import synth

    def get(i, walk_num=None):
        key = (i, walk_num)
        if key not in _CACHE:
            _CACHE[key] = synth.make_config(i, walk_num=walk_num)
        return _CACHE[key]
    return get


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle

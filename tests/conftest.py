import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def make_setup(p, **kw):
    from oracle.cell import Setup
    args = dict(lattice=p["lattice"], kmesh=p["kmesh"], ecut=p["ecut"], fft=p["fft"],
                nbands=p["nbands"], nocc=p["nocc"], A=p["A"], C=p["C"])
    args.update(kw)
    return Setup(**args)


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(12345)

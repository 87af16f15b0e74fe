import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MASTER_SEED = 20210103


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: full-size oracle work (tens of seconds)")


@pytest.fixture(scope="session")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def full_keys(O):
    """Oracle keys at the gate-bootstrapping parameter set (n=500, N=1024)."""
    return O.keygen(O.GATE_PARAMS, MASTER_SEED)


@pytest.fixture(scope="session")
def tiny_params(O):
    return O.Params(n=24, N=64, l=3, Bgbit=10, t=8, basebit=2,
                    sigma_lwe=2.0 ** -15, sigma_bk=9e-9)


@pytest.fixture(scope="session")
def tiny_keys(O, tiny_params):
    return O.keygen(tiny_params, 77)


def signed32(x):
    x = np.asarray(x, dtype=np.int64) & 0xFFFFFFFF
    return np.where(x >= 2 ** 31, x - 2 ** 32, x)

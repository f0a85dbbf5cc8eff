import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def si64():
    from tbinputs import si_system
    return si_system((2, 2, 2), sigma=0.05, seed=1, cutoff=4.0)


@pytest.fixture(scope="session")
def si64_dense(si64):
    from oracle import dense
    S = si64.dense_S()
    H = dense.ased_hamiltonian(S, si64.eps, si64.K, si64.orbital_atom())
    return H, S

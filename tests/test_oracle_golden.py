"""The oracle against its stored values in tests/golden/ (written by
tests/golden/make_golden.py, which calls only the oracle and the input
generators): an unintended change to the oracle's arithmetic shows here.
The stored values also carry the closed-form relations they must obey."""
import json
import os
import sys

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def stored():
    with open(os.path.join(GOLDEN, "si64.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def fresh():
    sys.path.insert(0, GOLDEN)
    try:
        import make_golden
    finally:
        sys.path.remove(GOLDEN)
    return make_golden.si64_values()


def test_oracle_reproduces_stored_values(stored, fresh):
    assert stored["columns"] == fresh["columns"] and stored["rows"] == fresh["rows"]
    for key in ("G_jj_re", "G_jj_im", "G_ij_re", "G_ij_im"):
        a, b = np.array(stored[key]), np.array(fresh[key])
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max(), key
    for key in ("mulliken", "lanczos_a", "lanczos_b"):
        assert np.allclose(stored[key], fresh[key], rtol=1e-12, atol=1e-12), key
    for key in ("band_energy", "electron_count", "lanczos_nrm2"):
        assert stored[key] == pytest.approx(fresh[key], rel=1e-12), key


def test_stored_values_obey_the_closed_forms(stored):
    """-Im G_jj(z) > 0 for Im z > 0 (a positive local density of states);
    the Lanczos coefficients have b_0 = 0 and b_n > 0, and e_j^T S^-1 e_j > 0."""
    assert np.all(np.array(stored["G_jj_im"]) < 0.0)
    b = np.array(stored["lanczos_b"])
    assert b[0] == 0.0 and np.all(b[1:] > 0.0)
    assert stored["lanczos_nrm2"] > 0.0

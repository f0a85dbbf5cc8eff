"""Host-side planning of the mixed path's Chebyshev corrections, without a
GPU: the spectrum bounds of S from the library's Lanczos run against dense
eigenvalues, and the step coefficients against the closed form of the
scaled Chebyshev polynomials they must reproduce."""
import math

import numpy as np
import pytest

from tbinputs import si_system, water_system


@pytest.fixture(scope="module")
def P():
    import paper_1002_1202_gb300 as pkg
    pkg.build()
    return pkg


@pytest.mark.parametrize("which", ["si64", "water8", "si512"])
def test_bounds_enclose_the_spectrum(P, which):
    s = {"si64": lambda: si_system((2, 2, 2), sigma=0.05, seed=1),
         "water8": lambda: water_system(8, seed=4, cutoff=3.0, excess_proton=False),
         "si512": lambda: si_system((4, 4, 4), seed=3)}[which]()
    ev = np.linalg.eigvalsh(s.dense_S())
    lo, hi = P.tb_overlap_bounds_desc(s)
    assert 0.0 < lo <= ev[0] and hi >= ev[-1]
    assert lo >= 0.9 * ev[0] and hi <= 1.05 * ev[-1]


def test_bounds_reject_indefinite_and_malformed(P):
    import dataclasses
    s = si_system((2, 2, 2), sigma=0.05, seed=1)
    sv = s.S_vals.copy()
    bo = s.block_offsets()
    for i in range(s.n_atoms):
        for b in range(s.brow_ptr[i], s.brow_ptr[i + 1]):
            if s.bcol[b] != i:
                sv[bo[b]:bo[b + 1]] *= 3.0
    assert np.linalg.eigvalsh(dataclasses.replace(s, S_vals=sv).dense_S())[0] < 0.0
    with pytest.raises(P.TBError) as e:
        P.tb_overlap_bounds_desc(dataclasses.replace(s, S_vals=sv))
    assert e.value.status == 3
    bc = s.bcol.copy()
    bc[3] = s.n_atoms + 2
    with pytest.raises(P.TBError) as e:
        P.tb_overlap_bounds_desc(dataclasses.replace(s, bcol=bc))
    assert e.value.status == 1


def _cheb(k, x):
    return np.cosh(k * np.arccosh(x)) if x >= 1.0 else np.cos(k * np.arccos(x))


@pytest.mark.parametrize("lo,hi", [(0.2, 2.4), (0.05, 3.0), (1.0, 1.5)])
def test_plan_step_counts(P, lo, hi):
    sigma = (hi - lo) / (hi + lo)
    for lo_tol, inner_tol in ((1e-6, 1e-12), (1e-6, 1e-13), (1e-5, 1e-12), (1e-6, 1e-7)):
        pl = P.tb_chebyshev_plan(lo, hi, lo_tol, inner_tol)
        n, nl, R = pl["n"], pl["n_last"], pl["rounds"]
        assert n % 2 == 1 and nl % 2 == 1 and 1 <= nl <= n
        assert 1.0 / _cheb(n, 1.0 / sigma) <= lo_tol
        assert n <= 2 or 1.0 / _cheb(n - 2, 1.0 / sigma) > lo_tol       # minimal up to the odd rounding
        assert R == math.ceil(math.log(inner_tol) / math.log(lo_tol) - 1e-9)
        # the planned rounds reach inner_tol by their bounds, with the last one's factor 2 to spare
        assert lo_tol ** (R - 1) / _cheb(nl, 1.0 / sigma) <= 0.5 * inner_tol * (1 + 1e-9) or nl == n
        assert pl["gamma"] == pytest.approx(2.0 / (lo + hi), rel=1e-7)
    assert P.tb_chebyshev_plan(-0.1, 2.0)["n"] == 0
    assert P.tb_chebyshev_plan(2.0, 2.0)["n"] == 0


def test_plan_coefficients_reproduce_chebyshev_polynomials(P):
    """Run the recurrence d_{k+1} = d_{k-1} + omega_k (gamma (f - A d_k) +
    d_k - d_{k-1}), d_0 = 0, d_1 = gamma f, with the plan's coefficients on a
    diagonal A with eigenvalues in [lo, hi]: the error of every component
    after k steps is p_k(lambda) = T_k((hi + lo - 2 lambda) / (hi - lo)) /
    T_k((hi + lo) / (hi - lo)), the scaled Chebyshev polynomial."""
    lo, hi = 0.2, 2.4
    pl = P.tb_chebyshev_plan(lo, hi, 1e-6, 1e-13)
    om, g = pl["omega"].astype(np.float64), pl["gamma"]
    lam = np.linspace(lo, hi, 41)
    f = np.ones_like(lam)
    x = f / lam
    dp, d = np.zeros_like(lam), g * f
    mu = (hi + lo) / (hi - lo)
    for k in range(1, pl["n"]):
        d, dp = dp + om[k] * (g * (f - lam * d) + d - dp), d
        err = (x - d) / x
        ref = np.array([_cheb(k + 1, (hi + lo - 2 * l) / (hi - lo)) for l in lam]) / _cheb(k + 1, mu)
        assert np.abs(err - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max()), k
    assert np.abs((x - d) / x).max() <= 1e-6


def test_bounds_and_plan_edge_cases(P):
    """One s atom (S = [1]) and one sp atom (S = I4, the Lanczos run stops
    at its first step): the bounds are the margins around 1 and the plan is
    short; malformed descriptions and tolerances are rejected."""
    import types
    one_s = types.SimpleNamespace(orb_per_atom=np.array([1]), brow_ptr=np.array([0, 1]), bcol=np.array([0]),
                                  S_vals=np.array([1.0]))
    one_sp = types.SimpleNamespace(orb_per_atom=np.array([4]), brow_ptr=np.array([0, 1]), bcol=np.array([0]),
                                   S_vals=np.eye(4).ravel())
    for sysm in (one_s, one_sp):
        lo, hi = P.tb_overlap_bounds_desc(sysm)
        assert lo == pytest.approx(0.97) and hi == pytest.approx(1.01)
        pl = P.tb_chebyshev_plan(lo, hi, 1e-6, 1e-12)
        assert 1 <= pl["n"] <= 9 and pl["rounds"] == 2
    bad = types.SimpleNamespace(orb_per_atom=np.array([2]), brow_ptr=np.array([0, 1]), bcol=np.array([0]),
                                S_vals=np.eye(2).ravel())
    with pytest.raises(P.TBError) as e:
        P.tb_overlap_bounds_desc(bad)
    assert e.value.status == 1
    for lo_tol, inner_tol in ((1.0, 1e-12), (0.0, 1e-12), (1e-6, 0.0)):
        with pytest.raises(P.TBError):
            P.tb_chebyshev_plan(0.2, 2.4, lo_tol, inner_tol)

"""Error statuses driven by host inputs (no device fault is involved).

A COCG breakdown (Section 3.3: alpha_n = rho_n / (p^T A p) needs a nonzero
denominator) is made on purpose with an isolated sp atom (S = 1, H = diag
of its levels) and the real seed shift z_0 = eps_s: then A(z_0) e_s = 0, so
mu = r'^T A p vanishes at the first step and the call must return
TB_ERR_BREAKDOWN.  eps_s = -13.5 is exact in FP32, so the double-float
products of the mixed path form the same exact zero where its inner solve
is exact."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TB_ERR_NOT_CONVERGED = 6
TB_ERR_BREAKDOWN = 7


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_1202_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope="module")
def atom(P):
    eps = np.array([-13.5, -6.5, -6.5, -6.5])
    return P.tb_create([4], [0, 1], [0], np.eye(4).ravel(), None, eps, 1.75)


def _opts(P, prec):
    if prec == "fp64":
        return P.tb_default_opts(precision=P.tb.TB_FP64)
    method = P.tb.TB_INNER_CG if prec == "mixed-cg" else P.tb.TB_INNER_CHEBYSHEV
    return P.tb_default_opts(precision=P.tb.TB_MIXED, inner_method=method)


@pytest.mark.parametrize("prec", ["fp64", "mixed-cg", "mixed"])
def test_breakdown_at_a_real_shift_on_a_level(P, atom, prec):
    """FP64 CG and the FP32 CG corrections solve S r' = e_s exactly for
    S = 1 (one CG step with alpha = 1), so mu is exactly zero and the call
    must report TB_ERR_BREAKDOWN.  The Chebyshev corrections solve it only
    to the inner tolerance, so mu is ~1e-12 instead of zero and the call may
    end either way the header allows for a real shift on a level: breakdown
    or no convergence."""
    opts = _opts(P, prec)
    z = np.array([-13.5 + 0.0j, -13.5 + 0.5j])
    with pytest.raises(P.TBError) as e:
        P.tb_shifted_cocg(atom, z, [0], opts=opts)
    if prec == "mixed":
        assert e.value.status in (TB_ERR_BREAKDOWN, TB_ERR_NOT_CONVERGED)
    else:
        assert e.value.status == TB_ERR_BREAKDOWN
    # the handle stays usable: away from the level the same column solves
    # to the closed form x = e_s / (z - eps_s)
    z2 = np.array([-13.0 + 0.5j])
    x, _ = P.tb_shifted_cocg(atom, z2, [0], opts=opts)
    X = x.cpu().numpy()[0, 0]
    want = np.zeros(4, dtype=complex)
    want[0] = 1.0 / (z2[0] + 13.5)
    assert np.abs(X - want).max() <= 1e-10

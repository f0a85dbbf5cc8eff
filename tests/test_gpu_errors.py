"""Error statuses driven by host inputs (no device fault is involved).

A COCG breakdown (Section 3.3: alpha_n = rho_n / (p^T A p) needs a nonzero
denominator) is made on purpose with an isolated sp atom (S = 1, H = diag
of its levels) and the real seed shift z_0 = eps_s: then A(z_0) e_s = 0, so
mu = r'^T A p vanishes at the first step and the call must return
TB_ERR_BREAKDOWN in both precisions.  eps_s = -13.5 is exact in FP32, so the
double-float products of the mixed path form the same exact zero."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_breakdown_at_a_real_shift_on_a_level(P, atom, prec):
    opts = P.tb_default_opts(precision=P.tb.TB_FP64 if prec == "fp64" else P.tb.TB_MIXED)
    z = np.array([-13.5 + 0.0j, -13.5 + 0.5j])
    with pytest.raises(P.TBError) as e:
        P.tb_shifted_cocg(atom, z, [0], opts=opts)
    assert e.value.status == TB_ERR_BREAKDOWN
    # the handle stays usable: away from the level the same column solves
    # to the closed form x = e_s / (z - eps_s)
    z2 = np.array([-13.0 + 0.5j])
    x, _ = P.tb_shifted_cocg(atom, z2, [0], opts=opts)
    X = x.cpu().numpy()[0, 0]
    want = np.zeros(4, dtype=complex)
    want[0] = 1.0 / (z2[0] + 13.5)
    assert np.abs(X - want).max() <= 1e-10

"""Pins of the exact-definition oracle (oracle.dense) against mathematics
other than itself: a second elimination algorithm, LAPACK, the spectral
decomposition, complex symmetry, the electron-count sum rule and the
extended-Hueckel dimer closed form."""
import math

import numpy as np
import pytest

from tbinputs import linspace_grid, build_system, H as HYD
from oracle import dense


def test_gauss_solve_vs_gauss_jordan_and_lapack():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(48, 48)) + 1j * rng.normal(size=(48, 48))
    B = rng.normal(size=(48, 5)) + 1j * rng.normal(size=(48, 5))
    X = dense.gauss_solve(A, B)
    assert np.abs(A @ X - B).max() < 1e-12
    assert np.abs(X - dense.gauss_jordan_inverse(A) @ B).max() < 1e-11
    assert np.abs(X - np.linalg.solve(A, B)).max() < 1e-11


def test_pivoting_needed():
    # zero leading entry: elimination without row exchange would divide by 0
    A = np.array([[0.0, 1.0], [1.0, 1.0]])
    x = dense.gauss_solve(A, np.array([1.0, 2.0]))
    assert np.allclose(x, [1.0, 1.0])


def test_green_vs_inverse_and_symmetry(si64_dense):
    H, S = si64_dense
    z = np.array([-7.3 + 0.01j, 1.2 + 0.01j])
    cols = [3, 77, 200]
    X = dense.green_columns(H, S, z, cols)
    for k, zk in enumerate(z):
        A = dense.shifted_matrix(H, S, zk)
        Ginv = dense.gauss_jordan_inverse(A)
        assert np.abs(X[k] - Ginv[:, cols]).max() < 1e-8 * np.abs(Ginv).max()
        # complex symmetry G_ij = G_ji (A(z)^T = A(z))
        for a, ca in enumerate(cols):
            for b, cb in enumerate(cols):
                assert abs(X[k][cb, a] - X[k][ca, b]) < 1e-9 * np.abs(X[k]).max()


def test_orthogonal_basis_reduces_to_spectral_form():
    # S = 1: G(z) = (z - H)^-1 = sum_m v_m v_m^T / (z - e_m)
    rng = np.random.default_rng(1)
    M = rng.normal(size=(40, 40))
    H = 0.5 * (M + M.T)
    e, V = np.linalg.eigh(H)
    z = 0.3 + 0.05j
    G = dense.green_columns(H, np.eye(40), [z], [0, 17])[0]
    ref = (V / (z - e)) @ V.T
    assert np.abs(G - ref[:, [0, 17]]).max() < 1e-10


def test_ased_dimer_closed_form():
    # two H atoms (one s orbital each): extended-Hueckel dimer, levels
    # eps (1 +/- K s) / (1 +/- s) for the overlap s
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.74]])
    sy = build_system([HYD, HYD], pos, np.array([50.0, 50.0, 50.0]), (False, False, False), 3.0, K=1.75)
    S = sy.dense_S()
    s = S[0, 1]
    H = dense.ased_hamiltonian(S, sy.eps, sy.K, sy.orbital_atom())
    ev = dense.generalized_eigvals(H, S)
    eps = sy.eps[0]
    want = sorted([eps * (1 + 1.75 * s) / (1 + s), eps * (1 - 1.75 * s) / (1 - s)])
    assert np.allclose(ev, want, rtol=1e-12, atol=1e-12)


def test_ased_structure(si64, si64_dense):
    H, S = si64_dense
    assert np.abs(H - H.T).max() == 0.0
    assert np.allclose(np.diag(H), si64.eps)
    oa = si64.orbital_atom()
    same = (oa[:, None] == oa[None, :]) & ~np.eye(len(S), dtype=bool)
    assert np.all(H[same] == 0.0)
    assert np.all((H != 0) <= ((S != 0) | np.eye(len(S), dtype=bool)))


def test_jacobi_vs_lapack():
    rng = np.random.default_rng(3)
    M = rng.normal(size=(30, 30))
    A = M + M.T
    assert np.abs(dense.jacobi_eigvals(A) - np.linalg.eigvalsh(A)).max() < 1e-11


def test_jacobi_stops_on_a_dominant_diagonal():
    """A matrix whose diagonal dominates its norm: the off-diagonal norm
    written as ||A||^2 - sum diag^2 cancels to ~sqrt(eps) ||A|| and never
    meets the tolerance; summed directly it does, and the eigenvalues agree
    with LAPACK."""
    rng = np.random.default_rng(0)
    # advance the generator past two other draws: with the matrix drawn
    # next, the cancelling form does not stop within 20 sweeps
    for n, scale in ((40, 1e3), (30, 1.0)):
        rng.uniform(-scale, scale, n)
        rng.standard_normal((n, n))
    A = np.diag(rng.uniform(-40.0, 40.0, 48)) + 0.1 * rng.standard_normal((48, 48))
    A = 0.5 * (A + A.T)
    ev = dense.jacobi_eigvals(A, max_sweeps=20)
    assert np.abs(ev - np.linalg.eigvalsh(A)).max() <= 1e-12 * np.abs(ev).max()


@pytest.mark.slow
def test_mulliken_sum_rule(si64, si64_dense):
    H, S = si64_dense
    z, w = linspace_grid(32)
    q = dense.mulliken_orbital(H, S, z, w, 2.0)
    eig = dense.generalized_eigvals(H, S)
    want = dense.electron_count_closed_form(eig, z, w, 2.0)
    assert abs(q.sum() - want) < 1e-8 * abs(want)
    # atom partition keeps the total
    qa = dense.mulliken_atom(q, si64.orbital_atom(), si64.n_atoms)
    assert abs(qa.sum() - q.sum()) < 1e-10


def test_mulliken_small_sum_rule_lapack():
    # sum rule on a small water cluster against LAPACK's generalized eigensolver
    import scipy.linalg as sl
    from tbinputs import water_box
    sp, pos, box, _ = water_box(3, seed=7, excess_proton=False)
    sy = build_system(sp, pos, box + 20.0, (False, False, False), 4.5)
    S = sy.dense_S()
    H = dense.ased_hamiltonian(S, sy.eps, sy.K, sy.orbital_atom())
    z, w = linspace_grid(9, -40.0, 5.0, 0.05)
    q = dense.mulliken_orbital(H, S, z, w)
    eig = sl.eigh(H, S, eigvals_only=True)
    assert abs(q.sum() - dense.electron_count_closed_form(eig, z, w)) < 1e-9


def _sparse_vs_dense(sy):
    """Eq. Hap-1 on the stored entries of S against the same rule applied
    to the dense S: the same formula with the same operands, so the two
    must agree bit for bit (any index slip in the COO walk shows up)."""
    S = sy.dense_S()
    oa = sy.orbital_atom()
    Hd = dense.ased_hamiltonian(S, sy.eps, sy.K, oa)
    Hs = dense.ased_hamiltonian_sparse(sy.to_csr(), sy.eps, sy.K, oa).toarray()
    assert Hs.shape == Hd.shape
    assert np.array_equal(Hs, Hd)
    return Hd


def test_ased_sparse_equals_dense_si64(si64):
    H = _sparse_vs_dense(si64)
    # the diagonal carries eps of the orbital itself (s and p levels differ)
    assert np.array_equal(np.diag(H), si64.eps)


def test_ased_sparse_equals_dense_water_ragged():
    """Water with the excess proton: O sp (4 orbitals) and H s (1 orbital)
    give 4x4, 4x1, 1x4 and 1x1 blocks and three different on-site levels, so
    the pairing eps[a] + eps[b] of the rule is checked across block shapes."""
    from tbinputs import water_box
    sp, pos, box, _ = water_box(6, seed=11, excess_proton=True)
    sy = build_system(sp, pos, box + 20.0, (False, False, False), 4.5)
    shapes = {(int(sy.orb_per_atom[i]), int(sy.orb_per_atom[j]))
              for i in range(sy.n_atoms) for j in sy.bcol[sy.brow_ptr[i]:sy.brow_ptr[i + 1]]}
    assert shapes == {(4, 4), (4, 1), (1, 4), (1, 1)}
    assert sy.n_orb == 6 * 6 + 1
    H = _sparse_vs_dense(sy)
    # an O s - H s element follows Eq. Hap-1 with the two different levels
    oa = sy.orbital_atom()
    S = sy.dense_S()
    o_s, h_s = 0, 4          # first O's s orbital, its first H
    assert oa[o_s] != oa[h_s]
    assert H[o_s, h_s] == sy.K * 0.5 * (sy.eps[o_s] + sy.eps[h_s]) * S[o_s, h_s] != 0.0

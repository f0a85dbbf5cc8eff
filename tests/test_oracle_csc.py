"""Pins of the charge-self-consistency oracle (Section 2.2, Eq. Hap-CSC)
against facts that do not come from the oracle itself:

* H^CSC is the derivative of the second-order energy E2 = 1/2 dq^T gamma dq
  with respect to the density matrix, through the Mulliken charges
  (finite differences of a quadratic: exact up to rounding);
* H^CSC is symmetric and vanishes at dq = 0;
* a uniform gamma (every entry c) adds c * sum(dq) * S to H, which moves every
  generalized eigenvalue by the same amount: the populations equal those of
  H0 at shifts z - c sum(dq), exactly;
* one atom with one s orbital: the self-consistent charge solves a scalar
  equation, found here by bisection on the closed-form population, an
  algorithm independent of the mixing loop;
* the loop's output is a fixed point: recomputing the populations from its
  dq with the dense definitions reproduces its q and meets the tolerance.
"""
import math

import numpy as np
import pytest

from tbinputs import water_system, klopman_ohno_gamma, valence_populations, gauss_legendre_grid
from oracle import dense, csc


@pytest.fixture(scope="module")
def water8():
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    S = s.dense_S()
    oa = s.orbital_atom()
    H0 = dense.ased_hamiltonian(S, s.eps, s.K, oa)
    return s, S, oa, H0


def test_correction_is_energy_derivative(water8):
    s, S, oa, H0 = water8
    rng = np.random.default_rng(7)
    N, n = S.shape[0], s.n_atoms
    gamma = klopman_ohno_gamma(s)
    q_ref = valence_populations(s)
    A = rng.standard_normal((N, N))
    rho = 0.5 * (A + A.T)
    B = rng.standard_normal((N, N))
    drho = 0.5 * (B + B.T)

    def E2(r):
        return csc.second_order_energy(gamma, csc.mulliken_charges_of_density(r, S, oa, n) - q_ref)

    h = 1e-3
    fd = (E2(rho + h * drho) - E2(rho - h * drho)) / (2 * h)
    dq = csc.mulliken_charges_of_density(rho, S, oa, n) - q_ref
    H1 = csc.csc_correction(S, oa, csc.csc_potential(gamma, dq))
    analytic = float(np.sum(H1 * drho.T))
    assert abs(fd - analytic) <= 1e-9 * max(1.0, abs(analytic))
    # a correction without the factor 1/2, or with S replaced by 1, fails
    assert abs(fd - 2 * analytic) > 1e-3 * abs(analytic)
    H1_noS = csc.csc_correction(np.ones_like(S), oa, csc.csc_potential(gamma, dq))
    assert abs(fd - float(np.sum(H1_noS * drho.T))) > 1e-3 * abs(analytic)


def test_correction_symmetric_and_zero_at_neutral(water8):
    s, S, oa, H0 = water8
    rng = np.random.default_rng(3)
    gamma = klopman_ohno_gamma(s)
    dq = rng.standard_normal(s.n_atoms) * 0.2
    H = csc.csc_hamiltonian(H0, S, oa, gamma, dq)
    assert np.array_equal(H, H.T)
    assert np.array_equal(csc.csc_hamiltonian(H0, S, oa, gamma, np.zeros(s.n_atoms)), H0)
    # on-site diagonal: eps + V_i (S_aa = 1)
    V = csc.csc_potential(gamma, dq)
    for a in range(S.shape[0]):
        assert abs(H[a, a] - (H0[a, a] + V[oa[a]])) <= 1e-12 * max(1.0, abs(H[a, a]))


def test_uniform_gamma_is_a_shift_of_the_energy_axis(water8):
    s, S, oa, H0 = water8
    rng = np.random.default_rng(5)
    c = 0.7
    gamma = np.full((s.n_atoms, s.n_atoms), c)
    dq = rng.standard_normal(s.n_atoms) * 0.3
    shift = c * dq.sum()
    z, w = gauss_legendre_grid(16, -40.0, -8.0, 1.0)
    q_csc = dense.mulliken_orbital(csc.csc_hamiltonian(H0, S, oa, gamma, dq), S, z, w)
    q_shift = dense.mulliken_orbital(H0, S, z - shift, w)
    assert np.abs(q_csc - q_shift).max() <= 1e-10


def _one_atom_population(E, z, w, g_s):
    # G = 1 / (z - E) for H = [[E]], S = [[1]]
    return -(g_s / math.pi) * float(np.sum(w / (z - E)).imag)


@pytest.mark.parametrize("U,eps,q_ref", [(5.0, -13.6, 1.0), (12.0, -9.0, 1.0), (3.0, -20.0, 0.0)])
def test_one_atom_loop_matches_bisection(U, eps, q_ref):
    z, w = gauss_legendre_grid(64, -40.0, -8.0, 2.0)
    g_s = 2.0

    def g(dq):   # strictly decreasing in dq for U > 0
        return _one_atom_population(eps + U * dq, z, w, g_s) - q_ref - dq

    lo, hi = -3.0, 3.0
    assert g(lo) > 0 > g(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            lo = mid
        else:
            hi = mid
    root = 0.5 * (lo + hi)
    out = csc.csc_loop(np.array([[eps]]), np.array([[1.0]]), np.array([0]), 1, np.array([[U]]),
                       np.array([q_ref]), z, w, g_s, mix=0.2, tol=1e-13, max_iter=2000)
    assert out["converged"]
    assert abs(out["dq"][0] - root) <= 1e-10


def test_water_loop_reaches_a_fixed_point(water8):
    s, S, oa, H0 = water8
    gamma = 0.25 * klopman_ohno_gamma(s)
    q_ref = valence_populations(s)
    z, w = gauss_legendre_grid(128, -60.0, -8.0, 2.0)
    out = csc.csc_loop(H0, S, oa, s.n_atoms, gamma, q_ref, z, w, mix=0.5, tol=1e-8, max_iter=60)
    assert out["converged"] and out["residual"] <= 1e-8
    # recompute the populations of the returned input with the dense definitions
    H = H0 + np.array([[0.5 * S[a, b] * (gamma[oa[a]] @ out["dq"] + gamma[oa[b]] @ out["dq"])
                        for b in range(S.shape[0])] for a in range(S.shape[0])])
    q = dense.mulliken_atom(dense.mulliken_orbital(H, S, z, w), oa, s.n_atoms)
    assert np.abs(q - out["q"]).max() <= 1e-10
    assert np.abs((q - q_ref) - out["dq"]).max() <= 1e-8
    # self-consistency changed the charges: the first iteration was far from it
    assert out["history"][0] > 1e-2


# ---------------------------------------------------------------------------
# forces of the charge-self-consistent model (contour grand potential Omega,
# free energy A(dq) = Omega(H0 + H^CSC(dq)) - V^T q_in + 1/2 dq^T gamma dq)
# ---------------------------------------------------------------------------
def test_grand_potential_gradients_match_differences(water8):
    s, S, oa, H0 = water8
    z, w = gauss_legendre_grid(64, -60.0, -8.0, 2.0)
    gH, gS = csc.grand_potential_gradients(H0, S, z, w)
    rng = np.random.default_rng(12)
    N = S.shape[0]
    mask = (np.abs(S) > 0).astype(float)
    for grad, which in ((gH, "H"), (gS, "S")):
        A = rng.standard_normal((N, N)) * mask
        D = 0.5 * (A + A.T)
        h = 1e-6
        if which == "H":
            fd = (csc.grand_potential(H0 + h * D, S, z, w) - csc.grand_potential(H0 - h * D, S, z, w)) / (2 * h)
        else:
            fd = (csc.grand_potential(H0, S + h * D, z, w) - csc.grand_potential(H0, S - h * D, z, w)) / (2 * h)
        assert abs(fd - float(np.sum(grad * D))) <= 1e-6 * max(1.0, abs(fd)), which
    # dOmega/dH is the density matrix itself (not the band-energy gradient)
    assert np.abs(gH - dense.density_matrix(H0, S, z, w).T).max() <= 1e-12


def test_grand_potential_sum_rule(water8):
    """d/dc Omega(H0 + c S) = Tr(rho S), the electron count, against the
    eigenvalue closed form of the sum rule."""
    s, S, oa, H0 = water8
    z, w = gauss_legendre_grid(64, -60.0, -8.0, 2.0)
    h = 1e-5
    fd = (csc.grand_potential(H0 + h * S, S, z, w) - csc.grand_potential(H0 - h * S, S, z, w)) / (2 * h)
    ne = dense.electron_count_closed_form(dense.generalized_eigvals(H0, S), z, w)
    assert abs(fd - ne) <= 1e-7 * ne


@pytest.fixture(scope="module")
def scc8(water8):
    s, S, oa, H0 = water8
    gamma = 0.25 * klopman_ohno_gamma(s)
    q_ref = valence_populations(s)
    z, w = gauss_legendre_grid(64, -60.0, -8.0, 2.0)
    out = csc.csc_loop(H0, S, oa, s.n_atoms, gamma, q_ref, z, w, mix=0.5, tol=1e-12, max_iter=300)
    assert out["converged"]
    return gamma, q_ref, z, w, out["dq"]


def test_scc_free_energy_is_stationary_at_self_consistency(water8, scc8):
    s, S, oa, H0 = water8
    gamma, q_ref, z, w, dq = scc8
    rng = np.random.default_rng(3)
    h = 1e-4

    def A(x):
        return csc.scc_free_energy(H0, S, oa, gamma, q_ref, x, z, w)

    # away from self-consistency dA/d dq = gamma (q_out - q_in) ...
    dq0 = np.zeros(s.n_atoms)
    q_out = dense.mulliken_atom(dense.mulliken_orbital(H0, S, z, w), oa, s.n_atoms)
    grad0 = gamma @ (q_out - (dq0 + q_ref))
    for _ in range(2):
        u = rng.standard_normal(s.n_atoms)
        fd = (A(dq0 + h * u) - A(dq0 - h * u)) / (2 * h)
        assert abs(fd - grad0 @ u) <= 1e-6 * max(1.0, abs(grad0 @ u))
    assert np.abs(grad0).max() > 1e-2
    # ... and it vanishes at the self-consistent dq
    for _ in range(2):
        u = rng.standard_normal(s.n_atoms)
        fd = (A(dq + h * u) - A(dq - h * u)) / (2 * h)
        assert abs(fd) <= 1e-7 * np.abs(grad0).max()


def test_scc_forces_match_differences(water8, scc8):
    """F = -dA/dR at self-consistency against central differences of A with
    the charges made self-consistent again at each displaced geometry (S,
    Eq. Hap-1 H0 and gamma rebuilt), zero net force, and a force without the
    Coulomb-gradient term failing."""
    from tbinputs import overlap_bond_derivatives, displaced, klopman_ohno_gamma_gradient
    s, S, oa, H0 = water8
    gamma, q_ref, z, w, dq = scc8
    dS = overlap_bond_derivatives(s)
    dg = 0.25 * klopman_ohno_gamma_gradient(s)
    F = csc.scc_forces(H0, S, oa, gamma, dg, q_ref, dq, z, w, dS, s.orb_per_atom, s.brow_ptr, s.bcol, s.eps, s.K)
    scale = np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() <= 1e-8 * scale
    h = 1e-4
    for atom, ax in ((2, 0), (9, 1)):
        As = []
        for sgn in (1, -1):
            sd = displaced(s, atom, ax, sgn * h)
            Sd = sd.dense_S()
            H0d = dense.ased_hamiltonian(Sd, sd.eps, sd.K, oa)
            gd = 0.25 * klopman_ohno_gamma(sd)
            out = csc.csc_loop(H0d, Sd, oa, s.n_atoms, gd, q_ref, z, w, mix=0.5, tol=1e-12, max_iter=300,
                               dq_init=dq)
            assert out["converged"]
            As.append(csc.scc_free_energy(H0d, Sd, oa, gd, q_ref, out["dq"], z, w))
        fd = -(As[0] - As[1]) / (2 * h)
        assert abs(F[atom, ax] - fd) <= 1e-5 * scale, (atom, ax, F[atom, ax], fd)
        F0 = csc.scc_forces(H0, S, oa, gamma, np.zeros_like(dg), q_ref, dq, z, w, dS, s.orb_per_atom, s.brow_ptr,
                            s.bcol, s.eps, s.K)
        assert abs(F0[atom, ax] - fd) > 1e-4 * scale

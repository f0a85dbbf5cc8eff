"""Pins of the oracle's z-derivatives and band-energy gradients against
facts that do not come from the oracle itself:

* dG/dz = -G S G against central differences of the dense solve in z
  (G is analytic in z off the real axis);
* the derivative recurrence of the method at a fixed step n (before
  convergence) against central differences of the method's own iterates in
  z_k, for a shift that never becomes the seed;
* the derivative at convergence, through seed switches, against -G S G;
* E = Tr(rho H) against the eigenvalue closed form
  -(g_s/pi) Im sum_k w_k sum_m eps_m / (z_k - eps_m);
* dE/dH and dE/dS against central differences of E under symmetric
  perturbations of H and of S;
* forces (chain rule through dE/dS, dE/dH and the geometry derivative of S)
  against central differences of E under atom displacements, and zero net
  force.
"""
import math

import numpy as np
import pytest

from tbinputs import si_system, water_system, linspace_grid
from oracle import dense, method


@pytest.fixture(scope="module")
def small():
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    return s, H, S


def test_dense_derivative_matches_differences(small):
    s, H, S = small
    z = np.array([-14.0 + 0.5j, -3.0 + 1.0j])
    cols = [0, 7]
    dG = dense.green_derivative_columns(H, S, z, cols)
    h = 1e-5
    fd = (dense.green_columns(H, S, z + h, cols) - dense.green_columns(H, S, z - h, cols)) / (2 * h)
    assert np.abs(dG - fd).max() <= 1e-6 * np.abs(dG).max()
    # a derivative missing S (-G G) fails
    G = dense.green_columns(H, S, z, cols)
    wrong = np.stack([-dense.green_matrix(H, S, zk) @ G[k] for k, zk in enumerate(z)])
    assert np.abs(wrong - fd).max() > 1e-3 * np.abs(dG).max()


@pytest.mark.parametrize("n", [3, 12, 30])
def test_method_derivative_recurrence_at_fixed_step(small, n):
    s, H, S = small
    z = np.array([-20.0 + 1.0j, -15.0 + 1.0j, -9.0 + 1.0j])
    j, k, h = 4, 2, 1e-6
    out = method.generalized_shifted_cocg(H, S, z, j, max_iter=n, switching=False, derivative=True)
    zp, zm = z.copy(), z.copy()
    zp[k] += h
    zm[k] -= h
    xp = method.generalized_shifted_cocg(H, S, zp, j, max_iter=n, switching=False)["x"][k]
    xm = method.generalized_shifted_cocg(H, S, zm, j, max_iter=n, switching=False)["x"][k]
    fd = (xp - xm) / (2 * h)
    assert np.abs(out["dx"][k] - fd).max() <= 1e-5 * np.abs(fd).max()
    # projected derivative equals the projection of the full derivative
    F = np.eye(S.shape[0])[[1, 4, 9]]
    outp = method.generalized_shifted_cocg(H, S, z, j, max_iter=n, switching=False, derivative=True,
                                           functionals=F, keep_full=False)
    assert np.abs(outp["dt"] - out["dx"] @ F.T).max() <= 1e-12 * np.abs(out["dx"]).max()


def test_method_derivative_converges_through_switches(small):
    s, H, S = small
    z, w = linspace_grid(12, -30.0, 0.0, 0.5)
    for j, force in ((2, 0), (11, 5)):
        out = method.generalized_shifted_cocg(H, S, z, j, tol=1e-12, derivative=True, force_switch_every=force)
        assert out["switches"] > 0
        ref = dense.green_derivative_columns(H, S, z, [j])[:, :, 0]
        assert np.abs(out["dx"] - ref).max() <= 1e-8 * np.abs(ref).max()


def test_band_energy_closed_form(small):
    s, H, S = small
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    E = dense.band_energy(H, S, z, w)
    eig = dense.generalized_eigvals(H, S)
    closed = -(2.0 / math.pi) * sum(wk * np.sum(eig / (zk - eig)) for zk, wk in zip(z, w)).imag
    assert abs(E - closed) <= 1e-9 * abs(closed)


def test_band_energy_gradients_match_differences(small):
    s, H, S = small
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    gH, gS = dense.band_energy_gradients(H, S, z, w)
    rng = np.random.default_rng(3)
    N = S.shape[0]
    mask = (np.abs(S) > 0).astype(float)          # perturb within the pattern
    for grad, which in ((gH, "H"), (gS, "S")):
        A = rng.standard_normal((N, N)) * mask
        D = 0.5 * (A + A.T)
        h = 1e-6
        if which == "H":
            fd = (dense.band_energy(H + h * D, S, z, w) - dense.band_energy(H - h * D, S, z, w)) / (2 * h)
        else:
            fd = (dense.band_energy(H, S + h * D, z, w) - dense.band_energy(H, S - h * D, z, w)) / (2 * h)
        analytic = float(np.sum(grad * D))
        assert abs(fd - analytic) <= 1e-6 * max(1.0, abs(analytic)), which


def test_forces_match_differences_of_energy(small):
    """F = -dE/dR by the chain rule through dE/dS, dE/dH and the geometry
    derivative of S, against central differences of the dense band energy
    of displaced systems (S and the Eq. Hap-1 H rebuilt)."""
    from tbinputs import overlap_bond_derivatives, displaced
    s, H, S = small
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    gH, gS = dense.band_energy_gradients(H, S, z, w)
    F = dense.forces_ased(gH, gS, overlap_bond_derivatives(s), s.orb_per_atom, s.brow_ptr, s.bcol, s.eps, s.K)
    assert np.abs(F.sum(axis=0)).max() <= 1e-8 * np.abs(F).max()      # no net force: translation invariance
    h = 1e-4
    for atom in (0, 5, 13):
        for ax in range(3):
            Es = []
            for sgn in (1, -1):
                sd = displaced(s, atom, ax, sgn * h)
                Sd = sd.dense_S()
                Es.append(dense.band_energy(dense.ased_hamiltonian(Sd, sd.eps, sd.K, sd.orbital_atom()), Sd, z, w))
            fd = -(Es[0] - Es[1]) / (2 * h)
            assert abs(F[atom, ax] - fd) <= 1e-5 * max(1.0, np.abs(F).max())


def test_mulliken_vjp_matches_differences(small):
    """dL/dH and dL/dS of L = sum_a v_a q_a against central differences of
    the dense Mulliken populations under symmetric perturbations."""
    s, H, S = small
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    rng = np.random.default_rng(8)
    N = S.shape[0]
    v = rng.standard_normal(N)
    gH, gS = dense.mulliken_vjp(H, S, z, w, v)
    mask = (np.abs(S) > 0).astype(float)

    def L(Hm, Sm):
        return float(v @ dense.mulliken_orbital(Hm, Sm, z, w))

    for grad, which in ((gH, "H"), (gS, "S")):
        A = rng.standard_normal((N, N)) * mask
        D = 0.5 * (A + A.T)
        h = 1e-6
        if which == "H":
            fd = (L(H + h * D, S) - L(H - h * D, S)) / (2 * h)
        else:
            fd = (L(H, S + h * D) - L(H, S - h * D)) / (2 * h)
        assert abs(fd - float(np.sum(grad * D))) <= 1e-6 * max(1.0, abs(fd)), which
    # v = 1 on every orbital: L is the electron count, whose H-gradient is
    # -(g_s/pi) Im sum_k w_k [G S G]^T = dE/dH of the energy with weights w_k / z_k
    gH1, _ = dense.mulliken_vjp(H, S, z, w, np.ones(N))
    gE, _ = dense.band_energy_gradients(H, S, z, w / z)
    assert np.abs(gH1 - gE).max() <= 1e-10 * np.abs(gE).max()

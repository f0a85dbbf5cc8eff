"""Charge self-consistency of the ASED Hamiltonian (TEST INFRASTRUCTURE).

Section 2.2, Eq. Hap-CSC: the charge-transfer correction to the Hamiltonian
is an extended Hubbard-type term,

    H^CSC_{i alpha, j beta} = 1/2 S_{i alpha, j beta} sum_k (gamma_ik + gamma_jk) dq_k
                            = 1/2 S_{i alpha, j beta} (V_i + V_j),   V = gamma dq,

where dq_k is the deviation of the Mulliken charge of atom k and gamma the
Coulomb interaction (chemical hardness on the diagonal).  The paper gives
neither the form of gamma nor the iteration that makes the charges
self-consistent; here gamma is an input matrix and the iteration is plain
linear mixing of dq, both choices stated in the function docstrings.

Everything is dense and plain: the populations come from
``dense.mulliken_orbital`` (exact Green's function by Gaussian elimination).
"""
from __future__ import annotations

import math

import numpy as np

from . import dense


def csc_potential(gamma: np.ndarray, dq: np.ndarray) -> np.ndarray:
    """V_i = sum_k gamma_ik dq_k (the sum inside Eq. Hap-CSC, one value per
    atom)."""
    gamma = np.asarray(gamma, dtype=np.float64)
    dq = np.asarray(dq, dtype=np.float64)
    n = len(dq)
    return np.array([sum(gamma[i, k] * dq[k] for k in range(n)) for i in range(n)])


def csc_correction(S: np.ndarray, orbital_atom: np.ndarray, V: np.ndarray) -> np.ndarray:
    """H^CSC of Eq. Hap-CSC: element (a, b) = 1/2 S_ab (V_{atom(a)} + V_{atom(b)})."""
    N = S.shape[0]
    out = np.zeros((N, N))
    for a in range(N):
        for b in range(N):
            out[a, b] = 0.5 * S[a, b] * (V[orbital_atom[a]] + V[orbital_atom[b]])
    return out


def csc_hamiltonian(H0: np.ndarray, S: np.ndarray, orbital_atom: np.ndarray, gamma: np.ndarray,
                    dq: np.ndarray) -> np.ndarray:
    """H = H0 + H^CSC(dq), H0 the charge-independent ASED Hamiltonian
    (Eq. Hap-1)."""
    return H0 + csc_correction(S, orbital_atom, csc_potential(gamma, dq))


def second_order_energy(gamma: np.ndarray, dq: np.ndarray) -> float:
    """E2 = 1/2 sum_ik gamma_ik dq_i dq_k: the second-order charge-transfer
    energy whose derivative with respect to the density matrix (through the
    Mulliken charges) is H^CSC.  Used to pin the correction, not by the
    loop."""
    n = len(dq)
    return 0.5 * sum(gamma[i, k] * dq[i] * dq[k] for i in range(n) for k in range(n))


def mulliken_charges_of_density(rho: np.ndarray, S: np.ndarray, orbital_atom: np.ndarray,
                                n_atoms: int) -> np.ndarray:
    """Atomic Mulliken populations q_i = sum_{alpha in i} (rho S)_{alpha alpha}
    of any density matrix rho."""
    N = S.shape[0]
    q_orb = np.array([sum(rho[a, b] * S[b, a] for b in range(N)) for a in range(N)])
    return dense.mulliken_atom(q_orb, orbital_atom, n_atoms)


def csc_loop(H0, S, orbital_atom, n_atoms, gamma, q_ref, z, w, g_s=2.0, *, mix=0.3, tol=1e-6,
             max_iter=100, dq_init=None):
    """Charge self-consistency by linear mixing (the paper names no mixing
    scheme).  Iteration m:

        H_m      = H0 + H^CSC(dq_in)
        q        = Mulliken populations of H_m (dense Green's function, the
                   quadrature z, w and spin factor g_s)
        dq_out   = q - q_ref
        res      = max_i |dq_out_i - dq_in_i|
        stop if res <= tol, else dq_in <- dq_in + mix (dq_out - dq_in)

    Returns a dict with the input dq of the last iteration (``dq``), the
    charges it produced (``q``), the iterations run, the final residual and
    the residual history.  ``converged`` is False when max_iter ran out
    (then ``dq`` and ``q`` are the last, unmixed pair)."""
    dq_in = np.zeros(n_atoms) if dq_init is None else np.array(dq_init, dtype=np.float64)
    hist = []
    for m in range(1, max_iter + 1):
        H = csc_hamiltonian(H0, S, orbital_atom, gamma, dq_in)
        q = dense.mulliken_atom(dense.mulliken_orbital(H, S, z, w, g_s), orbital_atom, n_atoms)
        dq_out = q - q_ref
        res = float(np.max(np.abs(dq_out - dq_in)))
        hist.append(res)
        if res <= tol or m == max_iter:
            return {"dq": dq_in, "q": q, "iterations": m, "residual": res, "history": hist,
                    "converged": res <= tol}
        dq_in = dq_in + mix * (dq_out - dq_in)


# --------------------------------------------------------------------------
# Forces of the charge-self-consistent model (reading: the paper cites the
# second-order expansion of the charge-transfer energy but prints no total
# energy).  With the quadrature z_k, w_k the occupation is a smeared step,
# so the functional whose exact derivative is the density matrix is the
# contour grand potential
#
#     Omega(H, S) = (g_s/pi) Im sum_k w_k Tr ln(z_k S - H),
#
# dOmega/dH_ab = rho_ba, rho = -(g_s/pi) Im sum_k w_k G(z_k).  The
# charge-self-consistent free energy
#
#     A(dq) = Omega(H0 + H^CSC(dq), S) - sum_i V_i (dq_i + q_ref_i) + 1/2 dq^T gamma dq,
#
# V = gamma dq, has dA/d dq = gamma (q_out - q_in): it is stationary at the
# self-consistent dq, so its forces need no charge response.
# --------------------------------------------------------------------------
def grand_potential(H, S, z, w, g_s=2.0) -> float:
    """Omega(H, S) = (g_s/pi) Im sum_k w_k Tr ln(z_k S - H) for real weights:
    det(z S - H) = det S prod_m (z - eps_m) with det S > 0, so the imaginary
    part is sum_m arg(z_k - eps_m), in (0, pi) for Im z_k > 0 (eps_m the
    generalized eigenvalues)."""
    eigs = dense.generalized_eigvals(H, S)
    tot = 0.0
    for zk, wk in zip(z, w):
        tot += float(np.real(wk)) * float(np.sum(np.angle(zk - eigs)))
    return (g_s / math.pi) * tot


def grand_potential_gradients(H, S, z, w, g_s=2.0):
    """dOmega/dH_ab = rho_ba and dOmega/dS_ab = (g_s/pi) Im sum_k w_k z_k G_ba(z_k)
    (d Tr ln M = Tr(M^-1 dM), M = z S - H), H_ab and S_ab independent
    entries.  Returns the two dense (N, N) real matrices."""
    rho = dense.density_matrix(H, S, z, w, g_s)
    WS = np.zeros(S.shape, dtype=np.complex128)
    for zk, wk in zip(z, w):
        WS += wk * zk * dense.green_matrix(H, S, zk)
    return rho.T.copy(), (g_s / math.pi) * WS.imag.T.copy()


def scc_free_energy(H0, S, orbital_atom, gamma, q_ref, dq, z, w, g_s=2.0) -> float:
    """A(dq) above: Omega of H = H0 + H^CSC(dq), minus the double-counted
    potential energy V^T (dq + q_ref), plus the second-order energy."""
    V = csc_potential(gamma, dq)
    H = H0 + csc_correction(S, orbital_atom, V)
    q_in = np.asarray(dq, dtype=np.float64) + np.asarray(q_ref, dtype=np.float64)
    return grand_potential(H, S, z, w, g_s) - float(V @ q_in) + second_order_energy(gamma, dq)


def scc_forces(H0, S, orbital_atom, gamma, dgamma, q_ref, dq, z, w, dS_dd, orb_per_atom, brow_ptr, bcol, eps, K,
               g_s=2.0) -> np.ndarray:
    """F_I = -dA/dR_I at a self-consistent dq (A stationary in dq), H0 by
    Eq. Hap-1 and gamma_ik depending on R_i - R_k:

        dA/dR = sum_ab rho_ba [dH0_ab/dR + 1/2 (V_a + V_b) dS_ab/dR]
                + sum_ab dOmega/dS_ab dS_ab/dR + 1/2 dq^T (dgamma/dR) dq,

    (the 1/2 S (dV_a + dV_b) part of dH^CSC/dR and -dV^T q_in cancel at
    self-consistency).  The first two lines are ``dense.forces_ased`` with
    gH = rho^T and gS = dOmega/dS + rho^T o 1/2 (V_a + V_b); the last adds
    -dq_I sum_k dgamma[I, k] dq_k, dgamma[I, k] = d gamma_Ik / d R_I.
    Returns (n_atoms, 3)."""
    V = csc_potential(gamma, dq)
    H = H0 + csc_correction(S, orbital_atom, V)
    gH, gS = grand_potential_gradients(H, S, z, w, g_s)
    N = S.shape[0]
    Vo = np.array([V[orbital_atom[a]] for a in range(N)])
    gS_eff = gS + gH * 0.5 * (Vo[:, None] + Vo[None, :])
    F = dense.forces_ased(gH, gS_eff, dS_dd, orb_per_atom, brow_ptr, bcol, eps, K)
    dq = np.asarray(dq, dtype=np.float64)
    for i in range(len(dq)):
        F[i] -= dq[i] * sum(dgamma[i, k] * dq[k] for k in range(len(dq)))
    return F

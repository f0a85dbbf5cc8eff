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

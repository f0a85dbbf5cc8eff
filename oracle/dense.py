"""Exact definitions in complex float64 (TEST INFRASTRUCTURE, see package doc).

Everything here is the plain definition written out, on dense matrices,
for systems small enough that O(N^3) work finishes in seconds.
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------------
# ASED Hamiltonian (Section 2.2)
# --------------------------------------------------------------------------
def ased_hamiltonian(S: np.ndarray, eps: np.ndarray, K: float, orbital_atom: np.ndarray) -> np.ndarray:
    """Dense ASED Hamiltonian.

    Section 2.2: the diagonal element H_{i alpha, i alpha} is the atomic
    level eps_{i alpha}; an element between orbitals of different atoms i != j
    follows Eq. (Hap-1), H = K * (H_{i alpha,i alpha} + H_{j beta,j beta}) / 2
    * S_{i alpha, j beta}, here with a constant K.  Two different orbitals on
    the same atom are orthogonal (their overlap is zero), so their element is
    zero as well.
    """
    N = len(eps)
    H = np.zeros((N, N))
    for a in range(N):
        for b in range(N):
            if a == b:
                H[a, b] = eps[a]
            elif orbital_atom[a] != orbital_atom[b]:
                H[a, b] = K * 0.5 * (eps[a] + eps[b]) * S[a, b]
    return H


def ased_hamiltonian_sparse(S_csr, eps: np.ndarray, K: float, orbital_atom: np.ndarray):
    """The same rule as ased_hamiltonian applied to the stored entries of a
    scipy.sparse overlap matrix (large systems; only the nonzero pattern of S
    can carry an off-diagonal element of Eq. Hap-1)."""
    import scipy.sparse as sp
    C = S_csr.tocoo()
    vals = np.zeros(C.nnz)
    for e in range(C.nnz):
        a, b = C.row[e], C.col[e]
        if a == b:
            vals[e] = eps[a]
        elif orbital_atom[a] != orbital_atom[b]:
            vals[e] = K * 0.5 * (eps[a] + eps[b]) * C.data[e]
    return sp.csr_matrix((vals, (C.row, C.col)), shape=S_csr.shape)


# --------------------------------------------------------------------------
# Linear solves (Eq. base-2, Eq. GreensFunc)
# --------------------------------------------------------------------------
def gauss_solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve A X = B by Gaussian elimination with partial pivoting.

    Forward elimination: at step k the row with the largest |A[p, k]|, p >= k,
    becomes the pivot row; multiples of it are subtracted from the rows below.
    Back substitution then runs from the last unknown to the first.
    """
    A = np.array(A, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    n = A.shape[0]
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if A[p, k] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        if p != k:
            A[[k, p]] = A[[p, k]]
            X[[k, p]] = X[[p, k]]
        f = A[k + 1:, k] / A[k, k]
        A[k + 1:, k:] -= f[:, None] * A[k, k:][None, :]
        X[k + 1:] -= f[:, None] * X[k][None, :]
    for k in range(n - 1, -1, -1):
        X[k] = (X[k] - A[k, k + 1:] @ X[k + 1:]) / A[k, k]
    return X[:, 0] if vec else X


def gauss_jordan_inverse(A: np.ndarray) -> np.ndarray:
    """Inverse of A by Gauss-Jordan elimination on [A | I] with partial
    pivoting: each pivot row is normalised and eliminated from every other
    row.  A second, independent route to A^-1 for brute-force checks."""
    A = np.array(A, dtype=np.complex128)
    n = A.shape[0]
    M = np.concatenate([A, np.eye(n, dtype=np.complex128)], axis=1)
    for k in range(n):
        p = k + int(np.argmax(np.abs(M[k:, k])))
        if M[p, k] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        M[[k, p]] = M[[p, k]]
        M[k] /= M[k, k]
        for i in range(n):
            if i != k and M[i, k] != 0:
                M[i] -= M[i, k] * M[k]
    return M[:, n:]


def shifted_matrix(H: np.ndarray, S: np.ndarray, z: complex) -> np.ndarray:
    """A(z) = z S - H: the matrix of Eq. (base-2) in a non-orthogonal basis
    ((E - H) becomes (E S - H) when <i|j> = S_ij)."""
    return z * S - H


def green_columns(H, S, z, cols) -> np.ndarray:
    """x_j(z_k) = (z_k S - H)^-1 e_j for every shift z_k and column j.

    Eq. (base-2) with |j> = e_j and Eq. (GreensFunc): G_ij(z) = <i|x^(j)>.
    Returns X with X[k, :, c] = x_{cols[c]}(z_k)  (shape K x N x len(cols)).
    """
    N = S.shape[0]
    cols = np.asarray(cols)
    B = np.zeros((N, len(cols)), dtype=np.complex128)
    B[cols, np.arange(len(cols))] = 1.0
    return np.stack([gauss_solve(shifted_matrix(H, S, zk), B) for zk in z])


def green_matrix(H, S, zk) -> np.ndarray:
    """Full G(z) = (z S - H)^-1 (all columns)."""
    N = S.shape[0]
    return gauss_solve(shifted_matrix(H, S, zk), np.eye(N, dtype=np.complex128))


# --------------------------------------------------------------------------
# Density matrix and Mulliken populations (Section 2.2)
# --------------------------------------------------------------------------
def density_matrix(H, S, z, w, g_s=2.0) -> np.ndarray:
    """rho = -(g_s / pi) Im sum_k w_k G(z_k): the energy-integrated Green's
    function (the paper integrates G into the charge density; the quadrature
    z_k, w_k is an input)."""
    rho = np.zeros(S.shape, dtype=np.complex128)
    for zk, wk in zip(z, w):
        rho += wk * green_matrix(H, S, zk)
    return -(g_s / math.pi) * rho.imag


def mulliken_orbital(H, S, z, w, g_s=2.0) -> np.ndarray:
    """Gross Mulliken population of every orbital, q_{i alpha} =
    (rho S)_{i alpha, i alpha} = sum_{j beta} rho_{i alpha, j beta} S_{j beta, i alpha}
    (the Mulliken partition of the overlap charge density, Section 2.2)."""
    rho = density_matrix(H, S, z, w, g_s)
    N = S.shape[0]
    return np.array([sum(rho[a, b] * S[b, a] for b in range(N)) for a in range(N)])


def mulliken_atom(q_orb: np.ndarray, orbital_atom: np.ndarray, n_atoms: int) -> np.ndarray:
    """Atomic gross population q_i = sum over the atom's orbitals."""
    q = np.zeros(n_atoms)
    for a, i in enumerate(orbital_atom):
        q[i] += q_orb[a]
    return q


# --------------------------------------------------------------------------
# Eigenvalues for the sum-rule closed form
# --------------------------------------------------------------------------
def cholesky(S: np.ndarray) -> np.ndarray:
    """Lower-triangular L with S = L L^T; raises if S is not positive
    definite (Section 3.3 relies on S being positive definite)."""
    n = S.shape[0]
    L = np.zeros_like(S, dtype=np.float64)
    for j in range(n):
        d = S[j, j] - L[j, :j] @ L[j, :j]
        if d <= 0.0:
            raise np.linalg.LinAlgError("overlap matrix is not positive definite")
        L[j, j] = math.sqrt(d)
        L[j + 1:, j] = (S[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def forward_substitution(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve L Y = B for lower-triangular L, row by row."""
    Y = np.array(B, dtype=np.float64)
    for i in range(L.shape[0]):
        Y[i] = (Y[i] - L[i, :i] @ Y[:i]) / L[i, i]
    return Y


def jacobi_eigvals(A: np.ndarray, tol: float = 1e-14, max_sweeps: int = 60) -> np.ndarray:
    """Eigenvalues of a real symmetric matrix by the cyclic Jacobi method:
    plane rotations annihilate the off-diagonal entries one pair at a time
    until the off-diagonal norm is below tol * ||A||_F."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    scale = np.linalg.norm(A)
    for _ in range(max_sweeps):
        # off-diagonal norm summed directly (the difference ||A||^2 - sum diag^2
        # cancels and cannot fall below ~sqrt(eps) ||A||)
        off = math.sqrt(float(np.sum(A * A, where=~np.eye(n, dtype=bool))))
        if off <= tol * scale:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if abs(apq) < 1e-300:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                rp = A[p].copy()
                rq = A[q].copy()
                A[p] = c * rp - s * rq
                A[q] = s * rp + c * rq
                cp = A[:, p].copy()
                cq = A[:, q].copy()
                A[:, p] = c * cp - s * cq
                A[:, q] = s * cp + c * cq
    else:
        raise RuntimeError("Jacobi eigensolver did not converge")
    return np.sort(np.diag(A))


def generalized_eigvals(H: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Eigenvalues eps_m of H c = eps S c, via S = L L^T and the symmetric
    matrix L^-1 H L^-T."""
    L = cholesky(S)
    Y = forward_substitution(L, H)            # L^-1 H
    C = forward_substitution(L, Y.T)          # L^-1 (L^-1 H)^T = L^-1 H L^-T
    return jacobi_eigvals(0.5 * (C + C.T))


def electron_count_closed_form(eigs: np.ndarray, z, w, g_s=2.0) -> float:
    """Sum rule: sum_{i alpha} q_{i alpha} = Tr(rho S)
    = -(g_s/pi) Im sum_k w_k Tr[(z_k S - H)^-1 S]
    = -(g_s/pi) Im sum_k w_k sum_m 1 / (z_k - eps_m),
    exact for any quadrature nodes and weights."""
    tot = 0.0 + 0.0j
    for zk, wk in zip(z, w):
        tot += wk * np.sum(1.0 / (zk - eigs))
    return -(g_s / math.pi) * tot.imag


# --------------------------------------------------------------------------
# z-derivatives and the band energy with its gradients (adjoint quantities)
# --------------------------------------------------------------------------
def green_derivative_columns(H, S, z, cols) -> np.ndarray:
    """dG/dz e_j = -G S G e_j for every shift (G = (zS - H)^-1, so
    dG/dz = -G (dA/dz) G with dA/dz = S); (K, N, R) complex."""
    N = S.shape[0]
    out = np.zeros((len(z), N, len(cols)), dtype=np.complex128)
    B = np.zeros((N, len(cols)), dtype=np.complex128)
    for c, j in enumerate(cols):
        B[j, c] = 1.0
    for k, zk in enumerate(z):
        A = shifted_matrix(H, S, zk)
        X = gauss_solve(A, B)
        out[k] = -gauss_solve(A, S @ X)
    return out


def band_energy(H, S, z, w, g_s=2.0) -> float:
    """Band-structure energy E = Tr(rho H) = sum_ab rho_ab H_ba with the
    energy-integrated density matrix rho of ``density_matrix``."""
    rho = density_matrix(H, S, z, w, g_s)
    return float(np.sum(rho * H.T))


def band_energy_gradients(H, S, z, w, g_s=2.0):
    """dE/dH_ab and dE/dS_ab, H_ab and S_ab taken as independent entries.
    With real weights E = -(g_s/pi) Im sum_k w_k z_k Tr[G_k S] for every H
    and S (because G (zS - H) = 1), and dG = G (dH - z dS) G, so
      dE/dH_ab = -(g_s/pi) Im sum_k w_k z_k [G S G]_ba,
      dE/dS_ab = -(g_s/pi) Im sum_k w_k (z_k G_ba - z_k^2 [G S G]_ba).
    Returns the two (N, N) real matrices."""
    N = S.shape[0]
    gH = np.zeros((N, N), dtype=np.complex128)
    gS = np.zeros((N, N), dtype=np.complex128)
    for zk, wk in zip(z, w):
        G = green_matrix(H, S, zk)
        GSG = G @ S @ G
        gH += wk * zk * GSG.T
        gS += wk * (zk * G.T - zk * zk * GSG.T)
    return -(g_s / math.pi) * gH.imag, -(g_s / math.pi) * gS.imag


def forces_ased(gH, gS, dS_dd, orb_per_atom, brow_ptr, bcol, eps, K) -> np.ndarray:
    """F_I = -dE/dR_I for H built by Eq. Hap-1 from S (charge-independent):
    every stored entry e of block (I, J), I != J, contributes
    v_e = (dE/dS_e + K (eps_a + eps_b) / 2 dE/dH_e) dS_e/dd with
    d = R_J - R_I, so F_I += v_e and F_J -= v_e (on-site H is eps, constant).
    gH, gS: dense (N, N) gradients; dS_dd: (3, n_values) in the block layout.
    Returns (n_atoms, 3)."""
    n = len(orb_per_atom)
    oo = np.concatenate([[0], np.cumsum(orb_per_atom)])
    F = np.zeros((n, 3))
    e = 0
    for i in range(n):
        for b in range(brow_ptr[i], brow_ptr[i + 1]):
            j = bcol[b]
            for a in range(orb_per_atom[i]):
                for c in range(orb_per_atom[j]):
                    ra, rb = oo[i] + a, oo[j] + c
                    if i != j:
                        wgt = gS[ra, rb] + 0.5 * K * (eps[ra] + eps[rb]) * gH[ra, rb]
                        F[i] += wgt * dS_dd[:, e]
                        F[j] -= wgt * dS_dd[:, e]
                    e += 1
    return F


def mulliken_vjp(H, S, z, w, v, g_s=2.0):
    """Vector-Jacobian product of the Mulliken populations: for
    L = sum_a v_a q_a (q_a the gross orbital populations, v_a weights per
    orbital), with D_v = diag(v) and dG = G (dH - z dS) G,
      dL/dH_ab = -(g_s/pi) Im sum_k w_k [G S D_v G]_ba,
      dL/dS_ab = -(g_s/pi) Im sum_k w_k (v_b G_ba - z_k [G S D_v G]_ba),
    H_ab, S_ab independent entries.  Returns the two (N, N) real matrices."""
    N = S.shape[0]
    Dv = np.diag(np.asarray(v, dtype=np.float64))
    gH = np.zeros((N, N), dtype=np.complex128)
    gS = np.zeros((N, N), dtype=np.complex128)
    for zk, wk in zip(z, w):
        G = green_matrix(H, S, zk)
        Gam = G @ S @ Dv @ G
        gH += wk * Gam.T
        gS += wk * ((Dv @ G).T - zk * Gam.T)
    return -(g_s / math.pi) * gH.imag, -(g_s / math.pi) * gS.imag

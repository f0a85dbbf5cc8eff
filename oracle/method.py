"""The method in the paper's order and notation (TEST INFRASTRUCTURE).

Section 3.3 (generalized shifted COCG) and Section 3.2 (generalized
Lanczos).  The matrices H (the Hamiltonian matrix, script-H in the paper) and
S only need to support ``@`` with a vector, so dense numpy arrays and
scipy.sparse matrices both work.

Problem orientation (reading of Eq. shift-E): the paper writes the seed system
as (S^-1 H + sigma_s) x = S^-1 b, i.e. (H + sigma_s S) x = b.  The Green's
function needs (z S - H) x = e_j, which is the same family with sigma = -z and
b = -e_j; this module works with A(z) = z S - H directly, so that
S^-1 A(z) = S^-1 A(z_s) + (z - z_s) * 1 and the shift of system k relative
to the seed is Delta_k = z_k - z_s.

Bilinear forms: COCG uses the unconjugated form u^T v (and u^T S v for the
S-product of Eq. 0.12); the conjugated 2-norm is only used for the
convergence test.

pi recurrence (Eq. shift:pi): the printed second term has a minus sign in
front of (beta_{n-1}/alpha_{n-1}) alpha_n (pi_n - pi_{n-1}).  Deriving the
recurrence from the seed residual polynomial gives a plus sign
(equivalently, a minus sign in front of (pi_{n-1} - pi_n)); the printed form
breaks the collinear-residual theorem (Eq. collinear) from the second step
on.  The derived sign is used here; ``pi_sign=-1`` reproduces the printed one.
"""
from __future__ import annotations

import math

import numpy as np


def cg_solve_real(S, b: np.ndarray, tol: float, max_iter: int):
    """Conjugate gradients for S x = b with real SPD S and a real right-hand
    side (Section 3.3: S is positive definite and close to the unit matrix, so
    r' = S^-1 r is obtained by CG).  Starts from x = 0 and stops when
    ||b - S x||_2 <= tol * ||b||_2.  Returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = math.sqrt(rr)
    if bnorm == 0.0:
        return x, 0
    it = 0
    while math.sqrt(rr) > tol * bnorm:
        if it >= max_iter:
            raise RuntimeError("inner CG did not converge")
        q = S @ p
        pq = float(p @ q)
        if pq <= 0.0:
            raise np.linalg.LinAlgError("overlap matrix is not positive definite")
        a = rr / pq
        x = x + a * p
        r = r - a * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def apply_S_inverse(S, r: np.ndarray, tol: float, max_iter: int):
    """r' = S^-1 r for a complex r: S is real, so the real and imaginary
    parts are two independent real CG solves."""
    xr, ir = cg_solve_real(S, np.ascontiguousarray(r.real), tol, max_iter)
    xi, ii = cg_solve_real(S, np.ascontiguousarray(r.imag), tol, max_iter)
    return xr + 1j * xi, max(ir, ii)


def generalized_shifted_cocg(H, S, z, j: int, *, tol=1e-10, inner_tol=1e-13, inner_max_iter=1000,
                             max_iter=100000, seed=0, switching=True, functionals=None,
                             keep_full=True, force_switch_every=0, pi_sign=1.0, record=False,
                             derivative=False):
    """Generalized shifted COCG for (z_k S - H) x_k = e_j, k = 0..K-1.

    Seed system (Eq. shift-E) solved by the recurrences Eq. (CGp:p),
    (CGp:x), (CGp:r) with r'_n = S^-1 r_n and
    alpha_n = rho_n / (p_n^T A(z_s) p_n),  beta_n = rho_{n+1} / rho_n,
    rho_n = r_n^T r'_n  (the S-products of the paper: (r', r')_S = r^T r').

    The seed direction p_n is not stored.  Because r_n = r_{n-1} -
    alpha_{n-1} A p_{n-1}, its product is A p_n = A r'_n + (beta_{n-1} /
    alpha_{n-1}) (r_{n-1} - r_n), and p_n^T A p_n = r'_n^T A p_n by
    A-conjugacy; so one product A(z_s) r'_n per step suffices and a seed
    switch is a rescaling of residuals only.

    Shifts (Eq. shift:pi, Eq. collinear): with Delta_k = z_k - z_s,
      pi^k_{n+1} = (1 + alpha_n Delta_k) pi^k_n
                   + pi_sign * (beta_{n-1} alpha_n / alpha_{n-1}) (pi^k_n - pi^k_{n-1}),
      r^k_n = r_n / pi^k_n,
      alpha^k_n = alpha_n pi^k_n / pi^k_{n+1},
      beta^k_n = beta_n (pi^k_n / pi^k_{n+1})^2,
      x^k_{n+1} = x^k_n + alpha^k_n p^k_n,
      p^k_{n+1} = r'_{n+1} / pi^k_{n+1} + beta^k_n p^k_n
    (only scalar-vector work per shift).  Shift k is converged when
    ||r_{n+1}||_2 / |pi^k_{n+1}| <= tol (||b|| = 1) and is frozen.

    Seed switching (Section 3.3, last paragraphs): when the seed has
    converged and other shifts have not, the unconverged shift s' with the
    largest residual becomes the seed.  Its residuals are r_n / pi^{s'}_n, so
    r_{n+1}, r'_{n+1}, r_n are divided by pi^{s'}_{n+1} (resp. pi^{s'}_n),
    rho_{n+1} by (pi^{s'}_{n+1})^2, every pi^k by pi^{s'}, and the seed
    scalars alpha_n, beta_n become alpha^{s'}_n, beta^{s'}_n.  Nothing of the
    Krylov history is discarded.

    ``functionals``: optional (M, N) array F; the result then carries
    t[k, m] = F[m] . x^k (the projected solution) tracked with scalars only.
    ``force_switch_every``: if > 0, switch to the worst unconverged shift
    every that many steps as well (used to exercise the switch).

    ``derivative``: also carry d/dz_k of every shift's iterates by
    differentiating the shift recurrences in z_k with the seed quantities
    (r_n, r'_n, alpha_n, beta_n and the switch rescalings) held fixed: only
    Delta_k = z_k - z_s depends on z_k, so
      dpi_{n+1} = alpha_n pi_n + (1 + alpha_n Delta) dpi_n
                  + (beta_{n-1} alpha_n / alpha_{n-1}) (dpi_n - dpi_{n-1}),
      d alpha^k = alpha_n (dpi_n pi_{n+1} - pi_n dpi_{n+1}) / pi_{n+1}^2,
      d beta^k  = 2 beta_n (pi_n / pi_{n+1}) (dpi_n pi_{n+1} - pi_n dpi_{n+1}) / pi_{n+1}^2,
      dx^k += d alpha^k p^k + alpha^k dp^k,
      dp^k  = -r'_{n+1} dpi_{n+1} / pi_{n+1}^2 + d beta^k p^k + beta^k dp^k,
    and a seed switch divides dpi, dpi_prev by the same constants as pi.  No
    extra matrix products: the derivative lives in the same Krylov sequence.
    The result then carries dx (K, N) and/or dt (K, M).

    Returns a dict with x (K, N) if keep_full, t (K, M) if functionals,
    conv_iter (K,), iterations, switches, and (if record) per-step histories.
    """
    z = np.asarray(z, dtype=np.complex128)
    K = len(z)
    N = S.shape[0]
    b = np.zeros(N, dtype=np.complex128)
    b[j] = 1.0
    F = None if functionals is None else np.asarray(functionals, dtype=np.complex128)

    s = int(seed)
    zs = z[s]
    r = b.copy()
    rp, m_in = apply_S_inverse(S, r, inner_tol, inner_max_iter)
    r_prev = np.zeros(N, dtype=np.complex128)
    rho = r @ rp
    alpha_prev, beta_prev = 1.0 + 0.0j, 0.0 + 0.0j
    pi = np.ones(K, dtype=np.complex128)
    pi_prev = np.ones(K, dtype=np.complex128)
    conv = np.zeros(K, dtype=bool)
    conv_iter = np.full(K, -1, dtype=np.int64)
    x = np.zeros((K, N), dtype=np.complex128) if keep_full else None
    p = np.tile(rp, (K, 1)) if keep_full else None
    t = np.zeros((K, F.shape[0]), dtype=np.complex128) if F is not None else None
    u = np.tile(F @ rp, (K, 1)) if F is not None else None
    hist = {"alpha": [], "beta": [], "rnorm": [], "seed": [], "pi": [], "inner": []} if record else None
    if derivative:
        dpi = np.zeros(K, dtype=np.complex128)
        dpi_prev = np.zeros(K, dtype=np.complex128)
        dx = np.zeros((K, N), dtype=np.complex128) if keep_full else None
        dp = np.zeros((K, N), dtype=np.complex128) if keep_full else None
        dt = np.zeros((K, F.shape[0]), dtype=np.complex128) if F is not None else None
        du = np.zeros((K, F.shape[0]), dtype=np.complex128) if F is not None else None
    switches = 0
    n = 0
    for n in range(max_iter):
        # seed step: A(z_s) p_n from the residuals, alpha_n, r_{n+1}
        q = zs * (S @ rp) - H @ rp
        Ap = q + (beta_prev / alpha_prev) * (r_prev - r)
        mu = rp @ Ap
        if mu == 0 or rho == 0:
            raise FloatingPointError("COCG breakdown")
        alpha = rho / mu
        r_new = r - alpha * Ap
        rp_new, m_in = apply_S_inverse(S, r_new, inner_tol, inner_max_iter)
        rho_new = r_new @ rp_new
        beta = rho_new / rho
        rnorm = float(np.linalg.norm(r_new))
        # shifts
        act = ~conv
        d = z - zs
        pi_new = pi.copy()
        pi_new[act] = (1.0 + alpha * d[act]) * pi[act] + \
            pi_sign * (beta_prev * alpha / alpha_prev) * (pi[act] - pi_prev[act])
        ak = np.zeros(K, dtype=np.complex128)
        bk = np.zeros(K, dtype=np.complex128)
        ak[act] = alpha * pi[act] / pi_new[act]
        bk[act] = beta * (pi[act] / pi_new[act]) ** 2
        if derivative:
            dpi_new = dpi.copy()
            dpi_new[act] = alpha * pi[act] + (1.0 + alpha * d[act]) * dpi[act] + \
                pi_sign * (beta_prev * alpha / alpha_prev) * (dpi[act] - dpi_prev[act])
            num = np.zeros(K, dtype=np.complex128)
            num[act] = (dpi[act] * pi_new[act] - pi[act] * dpi_new[act]) / pi_new[act] ** 2
            dak = alpha * num
            dbk = np.zeros(K, dtype=np.complex128)
            dbk[act] = 2.0 * beta * (pi[act] / pi_new[act]) * num[act]
            dip = np.zeros(K, dtype=np.complex128)
            dip[act] = -dpi_new[act] / pi_new[act] ** 2
            if keep_full:
                dx[act] += dak[act, None] * p[act] + ak[act, None] * dp[act]
                dp[act] = rp_new[None, :] * dip[act, None] + dbk[act, None] * p[act] + bk[act, None] * dp[act]
            if F is not None:
                fr_d = F @ rp_new
                dt[act] += dak[act, None] * u[act] + ak[act, None] * du[act]
                du[act] = fr_d[None, :] * dip[act, None] + dbk[act, None] * u[act] + bk[act, None] * du[act]
        if keep_full:
            x[act] += ak[act, None] * p[act]
            p[act] = rp_new[None, :] / pi_new[act, None] + bk[act, None] * p[act]
        if F is not None:
            fr = F @ rp_new
            t[act] += ak[act, None] * u[act]
            u[act] = fr[None, :] / pi_new[act, None] + bk[act, None] * u[act]
        res = np.full(K, np.inf)
        res[act] = rnorm / np.abs(pi_new[act])
        newly = act & (res <= tol)
        conv |= newly
        conv_iter[newly] = n + 1
        if record:
            hist["alpha"].append(alpha)
            hist["beta"].append(beta)
            hist["rnorm"].append(rnorm)
            hist["seed"].append(s)
            hist["pi"].append(pi_new.copy())
            hist["inner"].append(m_in)
        # advance n -> n+1
        pi_prev, pi = pi, pi_new
        if derivative:
            dpi_prev, dpi = dpi, dpi_new
        r_prev, r, rp, rho = r, r_new, rp_new, rho_new
        alpha_prev, beta_prev = alpha, beta
        if conv.all():
            break
        want = switching and (conv[s] or (force_switch_every > 0 and (n + 1) % force_switch_every == 0))
        if want:
            cand = np.where(conv, -1.0, res)
            s_new = int(np.argmax(cand))
            if s_new != s:
                c1, c0 = pi[s_new], pi_prev[s_new]
                r = r / c1
                rp = rp / c1
                r_prev = r_prev / c0
                rho = rho / (c1 * c1)
                alpha_prev, beta_prev = ak[s_new], bk[s_new]
                pi = pi / c1
                pi_prev = pi_prev / c0
                if derivative:
                    dpi = dpi / c1
                    dpi_prev = dpi_prev / c0
                zs = z[s_new]
                s = s_new
                switches += 1
    out = {"conv_iter": conv_iter, "iterations": n + 1, "switches": switches, "converged": bool(conv.all()),
           "seed": s}
    if keep_full:
        out["x"] = x
    if F is not None:
        out["t"] = t
    if derivative:
        if keep_full:
            out["dx"] = dx
        if F is not None:
            out["dt"] = dt
    if record:
        out["history"] = hist
    return out


def generalized_lanczos(H, S, j: int, n_steps: int, inner_tol=1e-13, inner_max_iter=1000):
    """Generalized Lanczos process for the operator S^-1 H (Section 3.2).

    Eq. (1.13): S^-1 H u^n = a_n u^n + b_{n+1} u^{n+1} + b_n u^{n-1}, b_0 = 0,
    with S-orthogonality (Eq. 1.18) (u^m, u^n)_S = u^m^T S u^n = delta_mn and
    b_n > 0.  The start vector is u^0 = S^-1 e_j / ||S^-1 e_j||_S, so that
    G_jj(z) = e_j^T (zS - H)^-1 e_j = nrm2 * [1 / (z - a_0 - b_1^2 / (z - a_1 - ...))]
    with nrm2 = e_j^T S^-1 e_j.

    a_n = (u^n, S^-1 H u^n)_S = u^n^T H u^n;
    w = S^-1 H u^n - a_n u^n - b_n u^{n-1};  b_{n+1} = ||w||_S;  u^{n+1} = w / b_{n+1}.
    Returns (a[n_steps], b[n_steps + 1] with b[0] = 0, nrm2).
    """
    N = S.shape[0]
    e = np.zeros(N)
    e[j] = 1.0
    v, _ = cg_solve_real(S, e, inner_tol, inner_max_iter)
    nrm2 = float(e @ v)
    u = v / math.sqrt(nrm2)
    u_prev = np.zeros(N)
    a = np.zeros(n_steps)
    b = np.zeros(n_steps + 1)
    for n in range(n_steps):
        hu = H @ u
        a[n] = float(u @ hu)
        y, _ = cg_solve_real(S, hu, inner_tol, inner_max_iter)
        w = y - a[n] * u - b[n] * u_prev
        bn = math.sqrt(max(0.0, float(w @ (S @ w))))
        b[n + 1] = bn
        if bn == 0.0:
            break
        u_prev, u = u, w / bn
    return a, b, nrm2


def lanczos_green(a, b, nrm2, z) -> np.ndarray:
    """G_jj(z) from the tridiagonal coefficients as a continued fraction
    (Section 3.2: the Green's function in the generalized Krylov subspace),
    evaluated from the bottom up."""
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    n = len(a)
    g = np.zeros_like(z)
    for m in range(n - 1, -1, -1):
        tail = b[m + 1] ** 2 * g if m + 1 < n else 0.0
        g = 1.0 / (z - a[m] - tail)
    return nrm2 * g

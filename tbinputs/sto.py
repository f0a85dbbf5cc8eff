"""Two-centre overlap integrals of normalised Slater-type orbitals (s and p).

The method works in a non-orthogonal local basis whose overlap matrix S is
built from "assumed atomic orbitals" with "STO parameters" (Section 2.2 and
Section 4.3 of the paper).  The paper gives no formulas for them, so this
module states the standard construction:

* radial part  R_n(r) = (2 zeta)^(n+1/2) / sqrt((2n)!) * r^(n-1) * exp(-zeta r)
  (normalised: int R^2 r^2 dr = 1), zeta in 1/bohr;
* real spherical harmonics  Y_s = 1/sqrt(4 pi),
  Y_p(axis) = sqrt(3/(4 pi)) * (unit vector . axis);
* bond-frame integrals ss, s-p(sigma), p(sigma)-s, pp(sigma), pp(pi) by
  Gauss quadrature in prolate spheroidal coordinates (lambda, mu, phi) with the
  two centres as foci; the integrand is a polynomial times an exponential in
  lambda, so Gauss-Laguerre in lambda and Gauss-Legendre in mu are exact up to
  rounding for the orders used here;
* Slater-Koster rotation to Cartesian p orbitals for a bond direction d.

This module is input generation only: it is shared by the oracle and the CUDA
path as the source of the synthetic overlap matrix and holds none of the
shifted-COCG arithmetic.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

BOHR_ANGSTROM = 0.529177210903  # 1 bohr in Angstrom


def radial_norm(n: int, zeta: float) -> float:
    """Normalisation constant of r^(n-1) exp(-zeta r)."""
    return (2.0 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n))


@lru_cache(maxsize=None)
def _nodes(n_lag: int, n_leg: int):
    t, wt = np.polynomial.laguerre.laggauss(n_lag)
    m, wm = np.polynomial.legendre.leggauss(n_leg)
    return t, wt, m, wm


def bond_integrals(n_a: int, zeta_a: float, n_b: int, zeta_b: float,
                   r_bohr, n_lag: int = 24, n_leg: int = 32) -> dict:
    """Overlaps of STOs on centre A (origin) and B (on +z at distance R).

    Both local z axes point from A to B.  ``r_bohr`` may be a scalar or a 1-D
    array of bond lengths.  Returns a dict with keys 'ss', 'sp' (s on A,
    p_sigma on B), 'ps' (p_sigma on A, s on B), 'pp_sigma', 'pp_pi'; each
    value has the shape of ``r_bohr``.

    With lambda = 1 + t / c, c = (R/2)(zeta_a + zeta_b), the lambda integrand
    is exp(-t) times a polynomial of degree <= n_a + n_b + 2 in t, so the
    Laguerre rule of order n_lag integrates it exactly; the mu integrand is a
    polynomial times exp(-(R/2)(zeta_a - zeta_b) mu), which the Legendre rule
    of order n_leg resolves to rounding for the exponents met here.
    """
    R = np.atleast_1d(np.asarray(r_bohr, dtype=np.float64))
    if np.any(R <= 0.0):
        raise ValueError("bond length must be positive")
    t, wt, mu, wm = _nodes(n_lag, n_leg)
    Rr = R[:, None, None]
    c = 0.5 * Rr * (zeta_a + zeta_b)
    L = 1.0 + t[None, :, None] / c          # lambda in [1, inf)
    M = mu[None, None, :]
    ra = 0.5 * Rr * (L + M)
    rb = 0.5 * Rr * (L - M)
    # exp(-za ra - zb rb) = exp(-c lambda) * exp(-(R/2)(za - zb) mu); the
    # exp(-c (lambda - 1)) part is the Laguerre weight.
    expo = np.exp(-c) * np.exp(-0.5 * Rr * (zeta_a - zeta_b) * M)
    weight = (wt[None, :, None] / c) * wm[None, None, :] * (0.5 * Rr) ** 3 * (L * L - M * M) * expo
    rad = radial_norm(n_a, zeta_a) * radial_norm(n_b, zeta_b) * ra ** (n_a - 1) * rb ** (n_b - 1)
    wr = weight * rad
    cos_a = (1.0 + L * M) / (L + M)
    cos_b = (L * M - 1.0) / (L - M)
    rho2 = (0.5 * Rr) ** 2 * (L * L - 1.0) * (1.0 - M * M)
    two_pi = 2.0 * math.pi
    ys = 1.0 / math.sqrt(4.0 * math.pi)
    yp = math.sqrt(3.0 / (4.0 * math.pi))
    out = {
        "ss": two_pi * ys * ys * wr.sum(axis=(1, 2)),
        "sp": two_pi * ys * yp * (wr * cos_b).sum(axis=(1, 2)),
        "ps": two_pi * yp * ys * (wr * cos_a).sum(axis=(1, 2)),
        "pp_sigma": two_pi * yp * yp * (wr * cos_a * cos_b).sum(axis=(1, 2)),
        # cos^2(phi) integrates to pi over a full turn
        "pp_pi": math.pi * yp * yp * (wr * rho2 / (ra * rb)).sum(axis=(1, 2)),
    }
    if np.ndim(r_bohr) == 0:
        return {k: float(v[0]) for k, v in out.items()}
    return out


def overlap_block(n_a: int, zeta_a: float, l_a: int,
                  n_b: int, zeta_b: float, l_b: int,
                  d_angstrom: np.ndarray) -> np.ndarray:
    """Overlap block <phi_{i alpha} | phi_{j beta}> for atom i at the origin
    and atom j at displacement d (Angstrom).

    l = 0 gives one s orbital; l = 1 gives s, px, py, pz (sp3 shell, both
    with the same n and zeta).  Returns an array of shape (n_orb_a, n_orb_b).
    """
    d = np.asarray(d_angstrom, dtype=np.float64)
    R = float(np.linalg.norm(d))
    u = d / R
    b = bond_integrals(n_a, zeta_a, n_b, zeta_b, R / BOHR_ANGSTROM)
    na_orb = 1 if l_a == 0 else 4
    nb_orb = 1 if l_b == 0 else 4
    blk = np.zeros((na_orb, nb_orb))
    blk[0, 0] = b["ss"]
    if l_b == 1:
        blk[0, 1:] = u * b["sp"]
    if l_a == 1:
        blk[1:, 0] = u * b["ps"]
    if l_a == 1 and l_b == 1:
        blk[1:, 1:] = np.outer(u, u) * b["pp_sigma"] + (np.eye(3) - np.outer(u, u)) * b["pp_pi"]
    return blk


def orbital_value(n: int, zeta: float, l: int, pts_bohr: np.ndarray) -> np.ndarray:
    """Values of the s (and px, py, pz if l=1) orbitals at points (bohr),
    shape (n_points, n_orb).  Used by the brute-force quadrature pins."""
    r = np.linalg.norm(pts_bohr, axis=-1)
    rad = radial_norm(n, zeta) * r ** (n - 1) * np.exp(-zeta * r)
    cols = [rad / math.sqrt(4.0 * math.pi)]
    if l == 1:
        with np.errstate(invalid="ignore", divide="ignore"):
            unit = np.where(r[..., None] > 0, pts_bohr / r[..., None], 0.0)
        for a in range(3):
            cols.append(rad * math.sqrt(3.0 / (4.0 * math.pi)) * unit[..., a])
    return np.stack(cols, axis=-1)

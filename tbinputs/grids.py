"""Energy points, quadrature weights and right-hand-side column choices.

The paper fixes no energy-integration rule.  Two grids are provided:
a uniform grid E_k = linspace(lo, hi, K) with trapezoid weights, and the
K-point Gauss-Legendre rule on [lo, hi]; in both z_k = E_k + i*eta.
"""
from __future__ import annotations

import numpy as np


def linspace_grid(K=32, lo=-20.0, hi=5.0, eta=0.01):
    E = np.linspace(lo, hi, K)
    w = np.full(K, (hi - lo) / (K - 1)) if K > 1 else np.ones(1)
    if K > 1:
        w[0] *= 0.5
        w[-1] *= 0.5
    return E + 1j * eta, w.astype(np.complex128)


def gauss_legendre_grid(K=256, lo=-20.0, hi=5.0, eta=0.01):
    x, w = np.polynomial.legendre.leggauss(K)
    E = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
    return E + 1j * eta, (0.5 * (hi - lo) * w).astype(np.complex128)


def choose_columns(N, R, seed=2):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=R, replace=False)).astype(np.int32)

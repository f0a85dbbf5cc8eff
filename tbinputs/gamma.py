"""Seeded inputs for the charge-self-consistent Hamiltonian: the Coulomb
interaction matrix gamma (eV per electron^2) and the reference populations.

The paper leaves the form of gamma open ("the Coulomb interaction between
atoms i and k or the chemical hardness", Section 2.2).  This generator uses
the Klopman-Ohno interpolation between an on-site hardness U and the bare
Coulomb law, gamma_ik = e^2 / sqrt(R_ik^2 + (e^2 / U_ik)^2) with
U_ik = (U_i + U_k) / 2 and minimum-image distances in periodic boxes; the
hardness values below are synthetic round numbers of the size quoted for
these elements in the tight-binding literature.
"""
from __future__ import annotations

import numpy as np

COULOMB_EV_ANGSTROM = 14.399645  # e^2 / (4 pi eps0) in eV * Angstrom

HARDNESS_EV = {"Si": 6.7, "O": 13.5, "H": 11.4}


def klopman_ohno_gamma(system, hardness=None) -> np.ndarray:
    """Dense (n_atoms, n_atoms) gamma of the system's atoms; gamma_ii = U_i."""
    hard = HARDNESS_EV if hardness is None else hardness
    U = np.array([hard[sp.name] for sp in system.species])
    pos = np.asarray(system.positions, dtype=np.float64)
    d = pos[:, None, :] - pos[None, :, :]
    box = np.asarray(system.box, dtype=np.float64)
    pbc = np.asarray(system.pbc, dtype=bool)
    for ax in range(3):
        if pbc[ax]:
            d[..., ax] -= box[ax] * np.round(d[..., ax] / box[ax])
    r2 = np.sum(d * d, axis=-1)
    Uik = 0.5 * (U[:, None] + U[None, :])
    return COULOMB_EV_ANGSTROM / np.sqrt(r2 + (COULOMB_EV_ANGSTROM / Uik) ** 2)


def valence_populations(system) -> np.ndarray:
    """Neutral-atom valence electron counts q_ref (Si 4, O 6, H 1)."""
    return np.array([float(sp.z_val) for sp in system.species])


def klopman_ohno_gamma_gradient(system, hardness=None) -> np.ndarray:
    """d gamma_ik / d R_i of ``klopman_ohno_gamma`` as an (n_atoms, n_atoms, 3)
    array: -e^2 (R_i - R_k) / (R_ik^2 + (e^2 / U_ik)^2)^(3/2), minimum image
    along periodic axes, zero on the diagonal (gamma_ii = U_i is constant).
    d gamma_ik / d R_k is its negative."""
    hard = HARDNESS_EV if hardness is None else hardness
    U = np.array([hard[sp.name] for sp in system.species])
    pos = np.asarray(system.positions, dtype=np.float64)
    d = pos[:, None, :] - pos[None, :, :]
    box = np.asarray(system.box, dtype=np.float64)
    pbc = np.asarray(system.pbc, dtype=bool)
    for ax in range(3):
        if pbc[ax]:
            d[..., ax] -= box[ax] * np.round(d[..., ax] / box[ax])
    r2 = np.sum(d * d, axis=-1)
    Uik = 0.5 * (U[:, None] + U[None, :])
    den = (r2 + (COULOMB_EV_ANGSTROM / Uik) ** 2) ** 1.5
    g = -COULOMB_EV_ANGSTROM * d / den[..., None]
    idx = np.arange(len(U))
    g[idx, idx, :] = 0.0
    return g

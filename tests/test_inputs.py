"""Pins of the synthetic-input generator (STO overlaps, geometry, block layout)."""
import math

import numpy as np
import pytest

from tbinputs import si_system, water_system
from tbinputs.sto import BOHR_ANGSTROM, bond_integrals, orbital_value, overlap_block
from oracle import dense


def _brute_overlap(na, za, la, nb, zb, lb, d_ang, npan=16, npts=8, ext=12.0):
    """Overlap block by composite Gauss-Legendre quadrature on a Cartesian
    box, with panel edges through both nuclei (independent of the prolate
    spheroidal rule used by the generator)."""
    d = np.asarray(d_ang) / BOHR_ANGSTROM
    xg, wg = np.polynomial.legendre.leggauss(npts)
    axes = []
    for ax in range(3):
        lo, hi = min(0.0, d[ax]) - ext, max(0.0, d[ax]) + ext
        brk = np.unique(np.concatenate([np.linspace(lo, hi, npan + 1), [0.0, d[ax]]]))
        pts = [0.5 * (b - a) * xg + 0.5 * (a + b) for a, b in zip(brk[:-1], brk[1:])]
        wts = [0.5 * (b - a) * wg for a, b in zip(brk[:-1], brk[1:])]
        axes.append((np.concatenate(pts), np.concatenate(wts)))
    (X, WX), (Y, WY), (Z, WZ) = axes
    out = None
    for i in range(len(X)):
        P = np.stack(np.meshgrid([X[i]], Y, Z, indexing="ij"), -1).reshape(-1, 3)
        w = (WX[i] * WY[:, None] * WZ[None, :]).ravel()
        part = (orbital_value(na, za, la, P) * w[:, None]).T @ orbital_value(nb, zb, lb, P - d)
        out = part if out is None else out + part
    return out


def test_1s1s_closed_form():
    # textbook overlap of two 1s STOs with equal exponent:
    # S = exp(-p) (1 + p + p^2/3), p = zeta R
    for R in (0.5, 1.4, 3.0, 7.0):
        p = 1.3 * R
        want = math.exp(-p) * (1 + p + p * p / 3)
        assert abs(bond_integrals(1, 1.3, 1, 1.3, R)["ss"] - want) < 1e-13


def test_same_centre_limit():
    # orbitals on (almost) the same centre: normalised and orthogonal
    b = bond_integrals(3, 1.6, 3, 1.6, 1e-4)
    assert abs(b["ss"] - 1) < 1e-6 and abs(b["pp_pi"] - 1) < 1e-6
    assert abs(b["pp_sigma"] + 1) > 1.9 - 1e-6 or abs(b["pp_sigma"] - 1) < 1e-6


@pytest.mark.parametrize("case", [
    ((3, 1.6, 1, 3, 1.6, 1), 2.35, 0),
    ((3, 1.6, 1, 3, 1.6, 1), 3.84, 1),
    ((2, 2.2, 1, 1, 1.3, 0), 0.96, 2),
    ((1, 1.3, 0, 2, 2.2, 1), 1.70, 3),
])
def test_overlap_block_vs_bruteforce(case):
    args, R, seed = case
    rng = np.random.default_rng(seed)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    got = overlap_block(*args, u * R)
    ref = _brute_overlap(*args, u * R)
    assert np.abs(got - ref).max() < 1e-7


@pytest.mark.parametrize("kind", ["si", "water"])
def test_overlap_matrix_properties(kind):
    sy = si_system() if kind == "si" else water_system(64, seed=4)
    S = sy.dense_S()
    assert np.abs(S - S.T).max() == 0.0
    assert np.allclose(np.diag(S), 1.0)
    oa = sy.orbital_atom()
    same = (oa[:, None] == oa[None, :]) & ~np.eye(len(S), dtype=bool)
    assert np.all(S[same] == 0.0)
    dense.cholesky(S)  # raises if S is not positive definite
    # block pattern: every block row holds its own diagonal block, columns sorted
    for i in range(sy.n_atoms):
        cols = sy.bcol[sy.brow_ptr[i]:sy.brow_ptr[i + 1]]
        assert i in cols and np.all(np.diff(cols) > 0)


def test_si_counts():
    sy = si_system()
    assert sy.n_atoms == 64 and sy.n_orb == 256
    # 4 first + 12 second neighbours + self under a 4.0 A cutoff
    assert 15 <= sy.nb / sy.n_atoms <= 17.5


def test_water_counts():
    sy = water_system(64, seed=4, excess_proton=True)
    assert sy.n_atoms == 3 * 64 + 1 and sy.n_orb == 6 * 64 + 1


def test_water_morton_order_is_a_permutation_of_molecules():
    """The Morton order lists the same molecules (each O followed by its own
    H atoms, the H3O+ kept whole) in a new order: the same atoms, the same
    overlap spectrum, and consecutive block rows that share more of their
    neighbour atoms."""
    a = water_system(100, seed=9)
    b = water_system(100, seed=9, order="morton")
    assert a.n_atoms == b.n_atoms and a.n_orb == b.n_orb
    key = lambda s: sorted((sp.name, *np.round(p, 10)) for sp, p in zip(s.species, s.positions))
    assert key(a) == key(b)
    # every H sits within O-H of the O that precedes it in the list
    for s in (a, b):
        o = None
        for sp, p in zip(s.species, s.positions):
            if sp.name == "O":
                o = p
            else:
                d = p - o
                d -= s.box * np.round(d / s.box)
                assert abs(np.linalg.norm(d) - 0.96) < 1e-9
    ea = np.linalg.eigvalsh(a.dense_S())
    eb = np.linalg.eigvalsh(b.dense_S())
    assert np.abs(ea - eb).max() <= 1e-12

    def distinct_ratio(s, G=16):
        d = r = 0
        for g0 in range(0, s.n_atoms, G):
            refs = s.bcol[s.brow_ptr[g0]:s.brow_ptr[min(s.n_atoms, g0 + G)]]
            d += len(set(refs.tolist()))
            r += len(refs)
        return d / r

    assert distinct_ratio(b) < distinct_ratio(a)


def test_cracked_slab_geometry():
    """The wedge-cracked Si slab: no atom centre (before displacement) inside
    the wedge, the gap 2 A wide at the tip and opening by 10 degrees, open
    along x and z, periodic along y; S symmetric and positive definite on a
    64-atom cut-out around the tip."""
    from tbinputs import si_cracked_slab, si_slab_system, cut_out
    sp, pos, box, pbc, tip = si_cracked_slab((6, 4, 6), sigma=0.0, seed=1)
    assert pbc == (False, True, False)
    assert len(pos) < 8 * 6 * 4 * 6
    x_tip, z_c = tip[0], tip[2]
    half = 1.0 + (x_tip - pos[:, 0]) * math.tan(math.radians(5.0))
    assert not np.any((pos[:, 0] < x_tip) & (np.abs(pos[:, 2] - z_c) < half))
    # atoms do remain just beyond the tip and beside the gap
    assert np.any((pos[:, 0] > x_tip) & (np.abs(pos[:, 2] - z_c) < 1.0))
    s = si_slab_system((6, 4, 6), seed=1)
    assert s.n_orb == 4 * s.n_atoms
    c = cut_out(s, s.meta["tip"], 64)
    assert c.n_atoms == 64 and c.pbc == (False, False, False)
    S = c.dense_S()
    assert np.allclose(S, S.T, atol=1e-14)
    assert np.linalg.eigvalsh(S)[0] > 0.0


def test_klopman_ohno_gradient_matches_differences():
    from tbinputs import klopman_ohno_gamma, klopman_ohno_gamma_gradient, displaced
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    g = klopman_ohno_gamma_gradient(s)
    h = 1e-5
    for atom, ax in ((0, 0), (5, 2)):
        fd = (klopman_ohno_gamma(displaced(s, atom, ax, h)) - klopman_ohno_gamma(displaced(s, atom, ax, -h))) / (2 * h)
        assert np.abs(fd[atom] - g[atom, :, ax]).max() <= 1e-7 * np.abs(g).max()
        assert np.abs(fd[:, atom] - g[atom, :, ax]).max() <= 1e-7 * np.abs(g).max()   # symmetric gamma
        others = np.arange(s.n_atoms) != atom
        assert np.abs(fd[np.ix_(others, others)]).max() == 0.0

"""Seeded synthetic tight-binding systems shaped like the paper's workloads.

The paper's own workloads (Au with the NRL Hamiltonian, Si fracture with the
Kwon Hamiltonian, proton transfer in water; Sections 3.4, 4.2, 4.3) need
parameter sets that are not available, so these generators stand in for them
with the same structure: Si in the diamond lattice with sp3 orbitals on every
atom (uniform 4x4 blocks) and liquid water with sp orbitals on O and s on H
(ragged 4x4 / 4x1 / 1x4 / 1x1 blocks).  All randomness comes from
``numpy.random.default_rng(seed)``.

The output is the block-sparse overlap matrix S in the layout the C-ABI
takes (atom block rows, full pattern, blocks row-major and concatenated),
the per-orbital on-site energies and the ASED constant K.  Building H from
them (Eq. Hap-1) is the method's job and is not done here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import cKDTree

from .sto import BOHR_ANGSTROM, bond_integrals


@dataclass(frozen=True)
class Species:
    name: str
    n: int          # principal quantum number of the STO shell
    zeta: float     # STO exponent, 1/bohr
    l: int          # 0: s only (1 orbital); 1: s + p (4 orbitals)
    eps: tuple      # on-site energies (eV): (eps_s,) or (eps_s, eps_p)
    z_val: int      # valence electrons (for charge deviations)

    @property
    def n_orb(self) -> int:
        return 1 if self.l == 0 else 4


SI = Species("Si", 3, 1.6, 1, (-13.55, -6.52), 4)
O = Species("O", 2, 2.2, 1, (-32.3, -14.8), 6)
H = Species("H", 1, 1.3, 0, (-13.6,), 1)
SPECIES = {s.name: s for s in (SI, O, H)}


@dataclass
class TBSystem:
    """A block-sparse non-orthogonal tight-binding system in atom order."""
    species: list                 # Species per atom
    positions: np.ndarray         # (n_atoms, 3) Angstrom
    box: np.ndarray               # (3,) Angstrom
    pbc: tuple                    # periodic flags per axis
    orb_per_atom: np.ndarray      # (n_atoms,) int32, 1 or 4
    brow_ptr: np.ndarray          # (n_atoms+1,) int64 block-row pointer
    bcol: np.ndarray              # (nb,) int32 block column (atom) index
    S_vals: np.ndarray            # concatenated row-major blocks, float64
    eps: np.ndarray               # (N,) on-site energies, eV
    K: float = 1.75               # ASED constant of Eq. Hap-1
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return len(self.orb_per_atom)

    @property
    def n_orb(self) -> int:
        return int(self.orb_per_atom.sum())

    @property
    def nb(self) -> int:
        return len(self.bcol)

    def orb_offset(self) -> np.ndarray:
        off = np.zeros(self.n_atoms + 1, dtype=np.int64)
        np.cumsum(self.orb_per_atom, out=off[1:])
        return off

    def block_offsets(self) -> np.ndarray:
        """Start of every block in S_vals (length nb+1)."""
        rows = np.repeat(np.arange(self.n_atoms), np.diff(self.brow_ptr))
        sizes = self.orb_per_atom[rows].astype(np.int64) * self.orb_per_atom[self.bcol]
        off = np.zeros(self.nb + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        return off

    def dense_S(self) -> np.ndarray:
        """Dense copy of S (orbital order); only for small systems."""
        N = self.n_orb
        oo = self.orb_offset()
        bo = self.block_offsets()
        S = np.zeros((N, N))
        for i in range(self.n_atoms):
            ni = self.orb_per_atom[i]
            for b in range(self.brow_ptr[i], self.brow_ptr[i + 1]):
                j = self.bcol[b]
                nj = self.orb_per_atom[j]
                S[oo[i]:oo[i] + ni, oo[j]:oo[j] + nj] = self.S_vals[bo[b]:bo[b + 1]].reshape(ni, nj)
        return S

    def to_csr(self):
        """S as a scipy.sparse CSR matrix in orbital order (format conversion)."""
        import scipy.sparse as sp
        oo = self.orb_offset()
        bo = self.block_offsets()
        rows = np.repeat(np.arange(self.n_atoms), np.diff(self.brow_ptr))
        ni = self.orb_per_atom[rows]
        nj = self.orb_per_atom[self.bcol]
        r_idx, c_idx = [], []
        for b in range(self.nb):
            a = np.arange(ni[b])[:, None]
            c = np.arange(nj[b])[None, :]
            r_idx.append(np.broadcast_to(oo[rows[b]] + a, (ni[b], nj[b])).ravel())
            c_idx.append(np.broadcast_to(oo[self.bcol[b]] + c, (ni[b], nj[b])).ravel())
        r_idx = np.concatenate(r_idx)
        c_idx = np.concatenate(c_idx)
        return sp.csr_matrix((self.S_vals.copy(), (r_idx, c_idx)), shape=(self.n_orb, self.n_orb))

    def orbital_atom(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_atoms), self.orb_per_atom)


def si_diamond(cells=(2, 2, 2), a=5.431, sigma=0.05, seed=1) -> tuple:
    """Diamond-lattice Si supercell, periodic, with Gaussian displacements of
    standard deviation ``sigma`` (Angstrom) per coordinate."""
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    frac = np.concatenate([base, base + 0.25])
    nx, ny, nz = cells
    grid = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    pos = (grid[:, None, :] + frac[None, :, :]).reshape(-1, 3) * a
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    box = np.array([nx, ny, nz], dtype=np.float64) * a
    return [SI] * len(pos), pos, box, (True, True, True)


def _morton_keys(p, L, bits=10):
    """Morton (Z-order) keys of positions in [0, L)^3: the cell indices on a
    2^bits grid with their bits interleaved."""
    q = np.clip((np.asarray(p) / L * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1)
    key = np.zeros(len(q), dtype=np.int64)
    for b in range(bits):
        for a in range(3):
            key |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return key


def water_box(n_mol: int, density=1.0, seed=4, excess_proton=True,
              r_oh=0.96, angle_deg=104.5, d_oo_min=2.5, order="placement") -> tuple:
    """Liquid-water-like box: O sites by random sequential placement with an
    O-O distance of at least ``d_oo_min``, random molecular orientations,
    rigid O-H = ``r_oh`` and H-O-H = ``angle_deg``.  With ``excess_proton``
    one molecule gets a third H (H3O+).  ``order``: molecules listed in
    their placement order, or ("morton") sorted by the Morton key of their
    O position, the spatial order a cell-list code keeps; the molecules and
    their geometry are the same either way."""
    if order not in ("placement", "morton"):
        raise ValueError(order)
    L = (n_mol * 18.015 / (0.60221408 * density)) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    ncell = max(1, int(L // d_oo_min))
    cell_sz = L / ncell
    cells = {}
    o_pos = []
    tries = 0
    while len(o_pos) < n_mol:
        tries += 1
        if tries > 200 * n_mol:
            raise RuntimeError("could not place water molecules")
        p = rng.uniform(0.0, L, size=3)
        c = tuple((p // cell_sz).astype(int) % ncell)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((c[0] + dx) % ncell, (c[1] + dy) % ncell, (c[2] + dz) % ncell)
                    for q in cells.get(key, ()):
                        d = p - q
                        d -= L * np.round(d / L)
                        if d @ d < d_oo_min ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            o_pos.append(p)
            cells.setdefault(c, []).append(p)
    half = math.radians(angle_deg) / 2.0
    local_h = np.array([[math.sin(half), 0.0, math.cos(half)],
                        [-math.sin(half), 0.0, math.cos(half)]]) * r_oh
    species, pos, first = [], [], []
    for m, p in enumerate(o_pos):
        first.append(len(species))
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        species.append(O)
        pos.append(p)
        hs = local_h @ rot.T
        for h in hs:
            species.append(H)
            pos.append(p + h)
        if excess_proton and m == 0:
            # third H opposite the bisector, tilted out of the molecular plane
            v = -(hs[0] + hs[1])
            v = v / np.linalg.norm(v) * math.cos(math.radians(20.0)) + rot[:, 1] * math.sin(math.radians(20.0))
            species.append(H)
            pos.append(p + r_oh * v / np.linalg.norm(v))
    pos = np.mod(np.array(pos), L)
    if order == "morton":
        first.append(len(species))
        perm = np.argsort(_morton_keys(np.mod(np.array(o_pos), L), L), kind="stable")
        idx = np.concatenate([np.arange(first[m], first[m + 1]) for m in perm])
        species = [species[i] for i in idx]
        pos = pos[idx]
    return species, pos, np.array([L, L, L]), (True, True, True)


def si_cracked_slab(cells=(10, 10, 10), a=5.431, tip_frac=0.5, tip_width=2.0, opening_deg=10.0, sigma=0.1,
                    seed=7) -> tuple:
    """Si slab with a wedge-shaped crack (a stand-in for the paper's Si
    fracture workload): the diamond lattice of ``cells`` cubic cells, periodic
    only along y (the crack front), open along x and z.  The crack enters
    from the x = 0 face at mid-height z_c and runs to the tip at
    x_tip = tip_frac * L_x; an atom is removed when x < x_tip and
    |z - z_c| < tip_width / 2 + (x_tip - x) tan(opening / 2), so the gap is
    ``tip_width`` wide at the tip and opens by ``opening_deg`` towards the
    mouth.  Then Gaussian displacements of ``sigma`` (Angstrom) per
    coordinate.  Returns (species, positions, box, pbc, tip) with tip the
    crack-tip point."""
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    frac = np.concatenate([base, base + 0.25])
    nx, ny, nz = cells
    grid = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    pos = (grid[:, None, :] + frac[None, :, :]).reshape(-1, 3) * a
    box = np.array([nx, ny, nz], dtype=np.float64) * a
    x_tip = tip_frac * box[0]
    z_c = 0.5 * box[2] - 0.125 * a          # between two atomic planes
    half = 0.5 * tip_width + (x_tip - pos[:, 0]) * math.tan(math.radians(0.5 * opening_deg))
    keep = ~((pos[:, 0] < x_tip) & (np.abs(pos[:, 2] - z_c) < half))
    pos = pos[keep]
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    tip = np.array([x_tip, 0.5 * box[1], z_c])
    return [SI] * len(pos), pos, box, (False, True, False), tip


def cut_out(system, center, n_atoms=64, cutoff=None) -> "TBSystem":
    """The ``n_atoms`` atoms of ``system`` nearest to ``center`` (minimum
    image along periodic axes) as an isolated cluster (no periodic axis),
    rebuilt with the same species, cutoff and K."""
    d = system.positions - np.asarray(center, dtype=np.float64)
    for ax in range(3):
        if system.pbc[ax]:
            d[:, ax] -= system.box[ax] * np.round(d[:, ax] / system.box[ax])
    idx = np.sort(np.argsort(np.einsum("ij,ij->i", d, d), kind="stable")[:n_atoms])
    pos = np.asarray(center, dtype=np.float64) + d[idx]
    sp = [system.species[i] for i in idx]
    cut = cutoff if cutoff is not None else system.meta.get("cutoff", 4.0)
    span = pos.max(0) - pos.min(0) + 2.0 * cut
    return build_system(sp, pos, span, (False, False, False), cut, system.K,
                        meta={"kind": "cut_out", "of": system.meta.get("kind"), "n_atoms": n_atoms, "cutoff": cut})


def _pairs(pos, box, pbc, cutoff):
    big = np.where(pbc, box, (pos.max(0) - pos.min(0)) + 4.0 * cutoff + 1.0)
    shifted = pos - np.where(pbc, 0.0, pos.min(0) - 2.0 * cutoff)
    shifted = np.where(pbc, np.mod(shifted, box), shifted)
    if np.any(np.asarray(pbc) & (box < 2.0 * cutoff)):
        raise ValueError("periodic box shorter than twice the cutoff")
    tree = cKDTree(shifted, boxsize=big)
    pairs = tree.query_pairs(cutoff, output_type="ndarray")
    d = pos[pairs[:, 1]] - pos[pairs[:, 0]]
    for ax in range(3):
        if pbc[ax]:
            d[:, ax] -= box[ax] * np.round(d[:, ax] / box[ax])
    return pairs, d


def bond_blocks(A, B, D) -> np.ndarray:
    """Overlap blocks <phi_A(0) | phi_B(d)> for bond vectors D (n, 3), Angstrom:
    STO bond integrals in the bond frame, Slater-Koster rotation (s, then p
    along x, y, z).  Returns (n, A.n_orb, B.n_orb)."""
    D = np.atleast_2d(np.asarray(D, dtype=np.float64))
    R = np.linalg.norm(D, axis=1)
    bi = bond_integrals(A.n, A.zeta, B.n, B.zeta, R / BOHR_ANGSTROM)
    u = D / R[:, None]
    blk = np.zeros((len(D), A.n_orb, B.n_orb))
    blk[:, 0, 0] = bi["ss"]
    if B.l == 1:
        blk[:, 0, 1:] = u * bi["sp"][:, None]
    if A.l == 1:
        blk[:, 1:, 0] = u * bi["ps"][:, None]
    if A.l == 1 and B.l == 1:
        uu = u[:, :, None] * u[:, None, :]
        blk[:, 1:, 1:] = uu * bi["pp_sigma"][:, None, None] + (np.eye(3)[None] - uu) * bi["pp_pi"][:, None, None]
    return blk


def overlap_bond_derivatives(system, h=1e-5) -> np.ndarray:
    """dS_e / dd for every stored entry e of S_vals, d = R_J - R_I the
    (minimum-image) bond vector of the entry's block (I, J), by central
    differences of ``bond_blocks`` (step h Angstrom); zero on diagonal
    blocks.  Returns (3, len(S_vals)).  Geometry input for forces: the
    derivative of the overlap with respect to the atom positions."""
    s = system
    pos = np.asarray(s.positions, dtype=np.float64)
    box = np.asarray(s.box, dtype=np.float64)
    bo = np.asarray(s.block_offsets())
    out = np.zeros((3, len(s.S_vals)))
    rows = np.repeat(np.arange(s.n_atoms), np.diff(s.brow_ptr))
    cols = np.asarray(s.bcol)
    off = np.flatnonzero(rows != cols)
    d = pos[cols[off]] - pos[rows[off]]
    for ax in range(3):
        if s.pbc[ax]:
            d[:, ax] -= box[ax] * np.round(d[:, ax] / box[ax])
    # one vectorised call per species pair and axis
    kind = {}
    for b, i, j in zip(off, rows[off], cols[off]):
        kind.setdefault((id(s.species[i]), id(s.species[j])), (s.species[i], s.species[j], []))[2].append(b)
    pos_in_off = np.empty(s.nb, dtype=np.int64)
    pos_in_off[off] = np.arange(len(off))
    for A, B, blocks in kind.values():
        blocks = np.asarray(blocks)
        D = d[pos_in_off[blocks]]
        n_e = A.n_orb * B.n_orb
        idx = bo[blocks][:, None] + np.arange(n_e)[None, :]
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            diff = (bond_blocks(A, B, D + e) - bond_blocks(A, B, D - e)) / (2 * h)
            out[ax, idx] = diff.reshape(len(blocks), n_e)
    return out


def displaced(system, atom, axis, delta):
    """The same system with one atom moved by delta (Angstrom) along an
    axis, rebuilt with the original cutoff (same blocks for small moves)."""
    s = system
    pos = np.array(s.positions, dtype=np.float64)
    pos[atom, axis] += delta
    return build_system(s.species, pos, s.box, s.pbc, s.meta.get("cutoff", 4.0), s.K, meta=s.meta)


def build_system(species, pos, box, pbc, cutoff, K=1.75, meta=None) -> TBSystem:
    """Overlap matrix in block-sparse form for atoms within ``cutoff``
    (Angstrom, minimum image along periodic axes)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = len(pos)
    pairs, d = _pairs(pos, np.asarray(box, dtype=np.float64), tuple(pbc), cutoff)
    # both triangles + diagonal
    I = np.concatenate([pairs[:, 0], pairs[:, 1], np.arange(n)])
    J = np.concatenate([pairs[:, 1], pairs[:, 0], np.arange(n)])
    D = np.concatenate([d, -d, np.zeros((n, 3))])
    order = np.lexsort((J, I))
    I, J, D = I[order], J[order], D[order]
    nb = len(I)
    orb = np.array([s.n_orb for s in species], dtype=np.int32)
    brow_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(brow_ptr, I + 1, 1)
    brow_ptr = np.cumsum(brow_ptr)
    sizes = orb[I].astype(np.int64) * orb[J]
    boff = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum(sizes, out=boff[1:])
    vals = np.zeros(boff[-1])
    sp_idx = np.array([list(SPECIES).index(s.name) for s in species])
    diag = I == J
    # diagonal blocks: normalised orbitals, same-atom s-p overlap vanishes
    for b in np.nonzero(diag)[0]:
        k = orb[I[b]]
        vals[boff[b]:boff[b + 1]] = np.eye(k).ravel()
    names = list(SPECIES)
    # compute the upper-triangle blocks and mirror them, so S is exactly symmetric
    keys = I.astype(np.int64) * n + J
    off = np.nonzero(I < J)[0]
    for ta in range(len(names)):
        for tb in range(len(names)):
            sel = off[(sp_idx[I[off]] == ta) & (sp_idx[J[off]] == tb)]
            if len(sel) == 0:
                continue
            A, B = SPECIES[names[ta]], SPECIES[names[tb]]
            for c0 in range(0, len(sel), 4096):
                ch = sel[c0:c0 + 4096]
                blk = bond_blocks(A, B, D[ch])
                na, nbo = A.n_orb, B.n_orb
                idx = boff[ch][:, None] + np.arange(na * nbo)[None, :]
                vals[idx] = blk.reshape(len(ch), -1)
                tr = np.searchsorted(keys, J[ch].astype(np.int64) * n + I[ch])
                idx_t = boff[tr][:, None] + np.arange(na * nbo)[None, :]
                vals[idx_t] = blk.transpose(0, 2, 1).reshape(len(ch), -1)
    eps = np.concatenate([[s.eps[0], s.eps[1], s.eps[1], s.eps[1]] if s.l == 1 else [s.eps[0]]
                          for s in species]).astype(np.float64)
    return TBSystem(species=list(species), positions=pos, box=np.asarray(box, dtype=np.float64),
                    pbc=tuple(pbc), orb_per_atom=orb, brow_ptr=brow_ptr, bcol=J.astype(np.int32),
                    S_vals=vals, eps=eps, K=K, meta=dict(meta or {}))


def si_system(cells=(2, 2, 2), sigma=0.05, seed=1, cutoff=4.0, K=1.75) -> TBSystem:
    sp, pos, box, pbc = si_diamond(cells, sigma=sigma, seed=seed)
    return build_system(sp, pos, box, pbc, cutoff, K,
                        meta={"kind": "si_diamond", "cells": list(cells), "sigma": sigma, "seed": seed,
                              "cutoff": cutoff})


def si_slab_system(cells=(10, 10, 10), sigma=0.1, seed=7, cutoff=4.0, K=1.75, **crack) -> TBSystem:
    """The cracked Si slab of ``si_cracked_slab`` as a system; the crack tip
    is in ``meta["tip"]``."""
    sp, pos, box, pbc, tip = si_cracked_slab(cells, sigma=sigma, seed=seed, **crack)
    return build_system(sp, pos, box, pbc, cutoff, K,
                        meta={"kind": "si_cracked_slab", "cells": list(cells), "sigma": sigma, "seed": seed,
                              "cutoff": cutoff, "tip": tip.tolist()})


def water_system(n_mol=64, seed=4, cutoff=4.5, K=1.75, excess_proton=True, order="placement") -> TBSystem:
    sp, pos, box, pbc = water_box(n_mol, seed=seed, excess_proton=excess_proton, order=order)
    return build_system(sp, pos, box, pbc, cutoff, K,
                        meta={"kind": "water", "n_mol": n_mol, "seed": seed, "cutoff": cutoff, "order": order})

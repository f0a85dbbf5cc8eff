"""z-derivatives of Green's function elements and the band energy with its
gradients and the forces they give on the GPU, against the oracle: the
dense definitions (-G S G, Tr(rho H), dE/dH, dE/dS, the chain rule to
forces) at convergence, the oracle's forward-differentiated recurrences after
a fixed number of steps, and energy differences of displaced geometries."""
import numpy as np
import pytest

from tbinputs import si_system, water_system, linspace_grid
from oracle import dense, method

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_1202_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope="module")
def si():
    s = si_system((2, 2, 2), sigma=0.05, seed=1)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    return s, H, S


def _rows(cols, rng, N):
    rows, ptr = [], [0]
    for j in cols:
        r = sorted(set([int(j)] + list(rng.choice(N, 6, replace=False))))
        rows += r
        ptr.append(len(rows))
    return np.array(ptr), np.array(rows)


def _dense_blocks(s, vals):
    """Values in the block layout of S_vals -> dense (N, N) matrix."""
    N = s.n_orb
    oo = s.orb_offset()
    bo = s.block_offsets()
    M = np.zeros((N, N))
    for i in range(s.n_atoms):
        ni = s.orb_per_atom[i]
        for b in range(s.brow_ptr[i], s.brow_ptr[i + 1]):
            j = s.bcol[b]
            nj = s.orb_per_atom[j]
            M[oo[i]:oo[i] + ni, oo[j]:oo[j] + nj] = vals[bo[b]:bo[b + 1]].reshape(ni, nj)
    return M


@pytest.mark.parametrize("prec,force", [(0, 0), (1, 0), (0, 5)], ids=["fp64", "mixed", "fp64-switches"])
def test_green_elements_dz_dense(P, si, prec, force):
    s, H, S = si
    z, w = linspace_grid(16, -20.0, 5.0, 1.0)
    cols = [3, 77, 200]
    ptr, rows = _rows(cols, np.random.default_rng(2), s.n_orb)
    h = P.tb_create_system(s)
    opts = P.tb_default_opts(precision=prec, force_switch_every=force)
    G, dG, st = P.tb_green_elements_dz(h, z, cols, ptr, rows, opts=opts)
    G, dG = G.cpu().numpy(), dG.cpu().numpy()
    Gd = dense.green_columns(H, S, z, cols)
    dGd = dense.green_derivative_columns(H, S, z, cols)
    for c in range(len(cols)):
        for m in range(ptr[c], ptr[c + 1]):
            assert np.abs(G[m] - Gd[:, rows[m], c]).max() <= 1e-7 * np.abs(Gd[:, :, c]).max()
            assert np.abs(dG[m] - dGd[:, rows[m], c]).max() <= 1e-6 * np.abs(dGd[:, :, c]).max()


def test_green_elements_dz_fixed_steps_match_method(P, si):
    s, H, S = si
    z, w = linspace_grid(16, -20.0, 5.0, 0.5)
    n = 25
    cols = [5, 130]
    ptr, rows = _rows(cols, np.random.default_rng(4), s.n_orb)
    h = P.tb_create_system(s)
    opts = P.tb_default_opts(max_iter=n, force_switch_every=7)
    G, dG, st = P.tb_green_elements_dz(h, z, cols, ptr, rows, opts=opts, allow_unconverged=True)
    dG = dG.cpu().numpy()
    for c, j in enumerate(cols):
        F = np.eye(s.n_orb)[rows[ptr[c]:ptr[c + 1]]]
        ref = method.generalized_shifted_cocg(H, S, z, j, max_iter=n, force_switch_every=7, derivative=True,
                                              functionals=F, keep_full=False)["dt"]
        got = dG[ptr[c]:ptr[c + 1]].T
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_band_energy_and_gradients(P, prec):
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    h = P.tb_create_system(s)
    E, gH, gS, st = P.tb_band_energy(h, z, w, opts=P.tb_default_opts(precision=prec), n_values=len(s.S_vals))
    assert st["status"] == "TB_OK"
    Ed = dense.band_energy(H, S, z, w)
    assert abs(E - Ed) <= 1e-8 * abs(Ed)
    gHd, gSd = dense.band_energy_gradients(H, S, z, w)
    mask = _dense_blocks(s, np.ones(len(s.S_vals))) > 0
    assert np.abs(_dense_blocks(s, gH)[mask] - gHd[mask]).max() <= 1e-7 * np.abs(gHd).max()
    assert np.abs(_dense_blocks(s, gS)[mask] - gSd[mask]).max() <= 1e-7 * np.abs(gSd).max()


def test_band_energy_of_a_batch(P):
    a = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    b = si_system((2, 2, 2), sigma=0.05, seed=1)
    z, w = linspace_grid(16, -40.0, 0.0, 1.0)
    hb = P.tb_create_batch([a, b])
    n_vals = len(a.S_vals) + len(b.S_vals)
    E, gH, gS, _ = P.tb_band_energy(hb, z, w, n_values=n_vals)
    Ea, gHa, gSa, _ = P.tb_band_energy(P.tb_create_system(a), z, w, n_values=len(a.S_vals))
    Eb, gHb, gSb, _ = P.tb_band_energy(P.tb_create_system(b), z, w, n_values=len(b.S_vals))
    assert abs(E - (Ea + Eb)) <= 1e-9 * abs(E)
    assert np.abs(gH - np.concatenate([gHa, gHb])).max() <= 1e-9 * np.abs(gH).max()
    assert np.abs(gS - np.concatenate([gSa, gSb])).max() <= 1e-9 * np.abs(gS).max()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_forces(P, prec):
    """Forces from the device band-energy gradients and the geometry
    derivatives of S: the oracle's chain rule on the dense gradients, the
    explicit-dH path, zero net force, and central differences of the dense
    band energy under atom displacements."""
    from tbinputs import overlap_bond_derivatives, displaced
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    h = P.tb_create_system(s)
    E, gH, gS, st = P.tb_band_energy(h, z, w, opts=P.tb_default_opts(precision=prec), n_values=len(s.S_vals))
    dS = overlap_bond_derivatives(s)
    F = P.tb_forces(h, gH, gS, dS)
    gHd, gSd = dense.band_energy_gradients(H, S, z, w)
    Fref = dense.forces_ased(gHd, gSd, dS, s.orb_per_atom, s.brow_ptr, s.bcol, s.eps, s.K)
    scale = np.abs(Fref).max()
    assert np.abs(F - Fref).max() <= 1e-7 * scale
    assert np.abs(F.sum(axis=0)).max() <= 1e-8 * scale
    # explicit dH/dd (the Eq. Hap-1 rule written out by the caller) gives the same forces
    oo = s.orb_offset()
    bo = s.block_offsets()
    rows = np.repeat(np.arange(s.n_atoms), np.diff(s.brow_ptr))
    dH = np.zeros_like(dS)
    for b in range(s.nb):
        i, j = rows[b], s.bcol[b]
        if i == j:
            continue
        ni, nj = s.orb_per_atom[i], s.orb_per_atom[j]
        c = 0.5 * s.K * (s.eps[oo[i]:oo[i] + ni][:, None] + s.eps[oo[j]:oo[j] + nj][None, :])
        dH[:, bo[b]:bo[b + 1]] = dS[:, bo[b]:bo[b + 1]] * c.ravel()[None, :]
    assert np.abs(P.tb_forces(h, gH, gS, dS, dH) - F).max() <= 1e-12 * scale
    # against differences of the energy of displaced geometries
    hstep = 1e-4
    for atom, ax in ((2, 0), (11, 2)):
        Es = []
        for sgn in (1, -1):
            sd = displaced(s, atom, ax, sgn * hstep)
            Sd = sd.dense_S()
            Es.append(dense.band_energy(dense.ased_hamiltonian(Sd, sd.eps, sd.K, sd.orbital_atom()), Sd, z, w))
        assert abs(F[atom, ax] + (Es[0] - Es[1]) / (2 * hstep)) <= 1e-5 * scale


def test_autograd_band_energy(P):
    """torch.autograd through the device adjoint: gradients equal
    tb_band_energy's, and a symmetric perturbation of S moves E by their
    contraction (central differences)."""
    import torch
    from paper_1002_1202_gb300.autograd import band_energy
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    # H in the block layout of S_vals
    oo, bo = s.orb_offset(), s.block_offsets()
    rows = np.repeat(np.arange(s.n_atoms), np.diff(s.brow_ptr))
    Hv = np.concatenate([H[oo[rows[b]]:oo[rows[b]] + s.orb_per_atom[rows[b]],
                           oo[s.bcol[b]]:oo[s.bcol[b]] + s.orb_per_atom[s.bcol[b]]].ravel() for b in range(s.nb)])
    Sv = torch.tensor(s.S_vals, dtype=torch.float64, requires_grad=True)
    Ht = torch.tensor(Hv, dtype=torch.float64, requires_grad=True)
    structure = (s.orb_per_atom, s.brow_ptr, s.bcol)
    E = band_energy(structure, Sv, Ht, z, w)
    E.backward()
    h = P.tb_create(s.orb_per_atom, s.brow_ptr, s.bcol, s.S_vals, Hv)
    E2, gH, gS, _ = P.tb_band_energy(h, z, w, n_values=len(s.S_vals))
    assert abs(E.item() - E2) <= 1e-12 * abs(E2)
    assert np.array_equal(Sv.grad.numpy(), gS) and np.array_equal(Ht.grad.numpy(), gH)
    # symmetric perturbation of S (block (i, j) and its transpose together)
    D = np.zeros_like(s.S_vals)
    b = int(s.brow_ptr[3]) + 1
    i, j = rows[b], s.bcol[b]
    t = int(np.nonzero((rows == j) & (s.bcol == i))[0][0])
    ni, nj = s.orb_per_atom[i], s.orb_per_atom[j]
    blk = np.random.default_rng(1).standard_normal((ni, nj))
    D[bo[b]:bo[b + 1]] = blk.ravel()
    D[bo[t]:bo[t + 1]] = blk.T.ravel()
    step = 1e-5
    Ep = band_energy(structure, torch.tensor(s.S_vals + step * D), Ht.detach(), z, w).item()
    Em = band_energy(structure, torch.tensor(s.S_vals - step * D), Ht.detach(), z, w).item()
    assert abs((Ep - Em) / (2 * step) - float(np.dot(gS, D))) <= 1e-5 * max(1.0, abs(float(np.dot(gS, D))))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_mulliken_vjp(P, prec):
    """dL/dH, dL/dS of L = sum_a v_a q_a from the device against the
    oracle's dense G S D_v G contraction, on every stored entry."""
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    v = np.random.default_rng(8).standard_normal(s.n_orb)
    h = P.tb_create_system(s)
    gH, gS, st = P.tb_mulliken_vjp(h, z, w, v, len(s.S_vals), opts=P.tb_default_opts(precision=prec))
    assert st["status"] == "TB_OK"
    gHd, gSd = dense.mulliken_vjp(H, S, z, w, v)
    mask = _dense_blocks(s, np.ones(len(s.S_vals))) > 0
    assert np.abs(_dense_blocks(s, gH)[mask] - gHd[mask]).max() <= 1e-7 * np.abs(gHd).max()
    assert np.abs(_dense_blocks(s, gS)[mask] - gSd[mask]).max() <= 1e-7 * np.abs(gSd).max()


def test_mulliken_vjp_chunks_and_device_weights(P, si):
    """A silicon cell (256 orbitals, so 4x4 blocks and many columns) with the
    weights v already on the device: the same contraction."""
    import torch
    s, H, S = si
    z, w = linspace_grid(8, -20.0, 5.0, 1.0)
    v = np.random.default_rng(3).standard_normal(s.n_orb)
    h = P.tb_create_system(s)
    gH, gS, _ = P.tb_mulliken_vjp(h, z, w, torch.tensor(v, device="cuda"), len(s.S_vals))
    gHd, gSd = dense.mulliken_vjp(H, S, z, w, v)
    mask = _dense_blocks(s, np.ones(len(s.S_vals))) > 0
    assert np.abs(_dense_blocks(s, gH)[mask] - gHd[mask]).max() <= 1e-7 * np.abs(gHd).max()
    assert np.abs(_dense_blocks(s, gS)[mask] - gSd[mask]).max() <= 1e-7 * np.abs(gSd).max()


# ---------------------------------------------------------------------------
# Si slab with a wedge crack (7680 atoms, N = 30720): the adjoint on a 64-atom
# cut-out around the crack tip against the dense oracle, and the Mulliken VJP
# of the full slab against central finite differences at 64 stored entries.
# Broadening 1 eV (the workload gives the shift count, 128, not eta).
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def slab():
    from tbinputs import si_slab_system
    return si_slab_system()


def _ased_block_values(s):
    """H of Eq. Hap-1 in the block layout of S_vals (4x4 blocks only)."""
    n, nb = s.n_atoms, s.nb
    assert np.all(s.orb_per_atom == 4)
    rows = np.repeat(np.arange(n), np.diff(s.brow_ptr))
    Sb = s.S_vals.reshape(nb, 4, 4)
    e = s.eps.reshape(n, 4)
    Hb = 0.5 * s.K * (e[rows][:, :, None] + e[s.bcol][:, None, :]) * Sb
    diag = rows == s.bcol
    Hb[diag] = np.einsum("bi,ij->bij", e[rows[diag]], np.eye(4))
    return Hb.reshape(-1)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_slab_cutout_adjoint_vs_dense(P, slab, prec):
    from tbinputs import cut_out, gauss_legendre_grid
    c = cut_out(slab, slab.meta["tip"], 64)
    S = c.dense_S()
    H = dense.ased_hamiltonian(S, c.eps, c.K, c.orbital_atom())
    z, w = gauss_legendre_grid(128, -20.0, 5.0, 1.0)
    h = P.tb_create_system(c)
    opts = P.tb_default_opts(precision=prec)
    E, gH, gS, st = P.tb_band_energy(h, z, w, opts=opts, n_values=len(c.S_vals))
    assert abs(E - dense.band_energy(H, S, z, w)) <= 1e-8 * abs(E)
    gHd, gSd = dense.band_energy_gradients(H, S, z, w)
    mask = _dense_blocks(c, np.ones(len(c.S_vals))) > 0
    assert np.abs(_dense_blocks(c, gH)[mask] - gHd[mask]).max() <= 1e-7 * np.abs(gHd).max()
    assert np.abs(_dense_blocks(c, gS)[mask] - gSd[mask]).max() <= 1e-7 * np.abs(gSd).max()
    # Mulliken VJP with weights on 8 orbitals (only their columns are solved)
    rng = np.random.default_rng(11)
    v = np.zeros(c.n_orb)
    v[rng.choice(c.n_orb, 8, replace=False)] = rng.standard_normal(8)
    vH, vS, _ = P.tb_mulliken_vjp(h, z, w, v, len(c.S_vals), opts=opts)
    rH, rS = dense.mulliken_vjp(H, S, z, w, v)
    assert np.abs(_dense_blocks(c, vH)[mask] - rH[mask]).max() <= 1e-7 * np.abs(rH).max()
    assert np.abs(_dense_blocks(c, vS)[mask] - rS[mask]).max() <= 1e-7 * np.abs(rS).max()


def test_slab_mixed_inner_solves_need_no_fp64_redo(P):
    """The band energy of a 4 x 4 x 4-cell cracked slab (480 atoms, all 1920
    columns, 128 shifts) in mixed precision: every inner solve reaches
    inner_tol on the mixed path.  Here lambda_min(S) = 0.146, so the
    double-float residual's own error (~2^-47 |S| |x|) can sit above
    inner_tol = 1e-13 for a column whose true residual is below; such a
    column must be settled by the FP64-checked spare rounds, not by an FP64
    CG redo of its panel (14 redos on this system before they existed)."""
    from tbinputs import si_slab_system, gauss_legendre_grid
    s = si_slab_system(cells=(4, 4, 4))
    z, w = gauss_legendre_grid(128, -20.0, 5.0, 1.0)
    h = P.tb_create_system(s)
    E, gH, gS, st = P.tb_band_energy(h, z, w, opts=P.tb_default_opts(tol=1e-8, precision=1),
                                     n_values=len(s.S_vals))
    assert st["unconverged"] == 0 and np.isfinite(E)
    assert st["inner_redos"] == 0, st


def _slab_vjp_finite_differences(P, s, n_each):
    """L = sum_a v_a q_a with weights on the 16 orbitals of the 4 atoms
    nearest the crack tip; dL/dH and dL/dS from the device VJP (mixed
    precision) at n_each stored H entries and n_each stored S entries of
    blocks within 6 A of the tip, each against a central difference
    (h = 1e-5) of L recomputed on the whole slab (FP64, outer tol 1e-12) with
    the entry and its transpose perturbed together.  Error bound: the central
    difference's truncation (O(h^2)) plus 2 eps / (2 h) for populations
    accurate to eps = 1e-12 sum |v|; asserted: 1e-5 of the largest gradient
    plus that rounding term.  Every solve is capped at 5000 outer
    iterations.  128 Gauss-Legendre shifts on [-20, 5] eV + 1i eV."""
    from tbinputs import gauss_legendre_grid
    z, w = gauss_legendre_grid(128, -20.0, 5.0, 1.0)
    tip = np.asarray(s.meta["tip"])
    d = s.positions - tip
    d[:, 1] -= s.box[1] * np.round(d[:, 1] / s.box[1])
    near = np.argsort(np.einsum("ij,ij->i", d, d))
    sup_atoms = near[:4]
    sup = np.concatenate([4 * a + np.arange(4) for a in sup_atoms]).astype(np.int32)
    rng = np.random.default_rng(5)
    v = np.zeros(s.n_orb)
    v[sup] = rng.standard_normal(len(sup))
    Hv = _ased_block_values(s)
    h0 = P.tb_create(s.orb_per_atom, s.brow_ptr, s.bcol, s.S_vals, Hv)
    gH, gS, st = P.tb_mulliken_vjp(h0, z, w, v, len(s.S_vals), opts=P.tb_default_opts(precision=1, max_iter=5000))
    assert st["status"] == "TB_OK"
    cols = np.sort(sup)
    fd_opts = P.tb_default_opts(precision=0, tol=1e-12, inner_tol=1e-13, max_iter=5000)

    def L(Svals, Hvals):
        hh = P.tb_create(s.orb_per_atom, s.brow_ptr, s.bcol, Svals, Hvals)
        q, _ = P.tb_mulliken_orbital(hh, z, w, cols, 2.0, opts=fd_opts)
        hh.close()
        return float(np.dot(v[cols], q.cpu().numpy()))

    # stored entries of blocks (I, J), I != J, with both atoms within 6 A of the tip
    rows = np.repeat(np.arange(s.n_atoms), np.diff(s.brow_ptr))
    r2 = np.einsum("ij,ij->i", d, d)
    cand = np.nonzero((rows != s.bcol) & (r2[rows] < 36.0) & (r2[s.bcol] < 36.0))[0]
    blocks = rng.choice(cand, 2 * n_each, replace=False)
    step = 1e-5
    errs, scale = [], max(np.abs(gH).max(), np.abs(gS).max())
    for k, b in enumerate(blocks):
        i, j = rows[b], s.bcol[b]
        t = int(np.nonzero((rows == j) & (s.bcol == i))[0][0])
        ai, bj = rng.integers(0, 4, size=2)
        e, et = 16 * b + 4 * ai + bj, 16 * t + 4 * bj + ai
        which = "H" if k < n_each else "S"
        D = np.zeros(len(s.S_vals))
        D[e] += 1.0
        D[et] += 1.0
        if which == "H":
            fd = (L(s.S_vals, Hv + step * D) - L(s.S_vals, Hv - step * D)) / (2 * step)
            an = gH[e] + gH[et]
        else:
            fd = (L(s.S_vals + step * D, Hv) - L(s.S_vals - step * D, Hv)) / (2 * step)
            an = gS[e] + gS[et]
        errs.append((abs(fd - an), abs(an), which, fd, an))
    worst = max(errs)
    assert worst[0] <= 1e-5 * scale + 2e-12 * np.abs(v).sum() / (2 * step), worst


def test_small_slab_mulliken_vjp_finite_differences(P):
    """The finite-difference check of the cracked-slab workload at a bounded
    size that runs by default: the same crack (2 A wide at the tip, opening
    10 degrees, 0.1 A displacements) in a slab of 5 x 5 x 5 diamond cells
    (1000 sites before the crack is cut), 8 H and 8 S entries near the tip."""
    from tbinputs import si_slab_system
    _slab_vjp_finite_differences(P, si_slab_system(cells=(5, 5, 5)), 8)


@pytest.mark.slow
@pytest.mark.skipif(not __import__("os").environ.get("TB_SLAB_FD"),
                    reason="128 full-slab solves; run with TB_SLAB_FD=1")
def test_slab_mulliken_vjp_finite_differences(P, slab):
    """The full cracked slab (10 x 10 x 10 cells, 7680 atoms): 32 H and 32 S
    entries (opt-in: 128 full-slab solves)."""
    _slab_vjp_finite_differences(P, slab, 32)


def _block_values(s, M):
    """The entries of a dense (N, N) matrix at the stored positions of the
    block layout of S_vals (the inverse of _dense_blocks on the pattern)."""
    oo = s.orb_offset()
    bo = s.block_offsets()
    out = np.zeros(len(s.S_vals))
    for i in range(s.n_atoms):
        ni = s.orb_per_atom[i]
        for b in range(s.brow_ptr[i], s.brow_ptr[i + 1]):
            j = s.bcol[b]
            nj = s.orb_per_atom[j]
            out[bo[b]:bo[b + 1]] = M[oo[i]:oo[i] + ni, oo[j]:oo[j] + nj].ravel()
    return out


@pytest.mark.parametrize("per_orbital", [False, True], ids=["atoms", "orbitals"])
def test_mulliken_autograd_function(P, per_orbital):
    """The torch.autograd Function of the Mulliken populations: forward
    against the oracle's dense populations, backward (a random incoming
    gradient) against the dense G S D_v G contraction with v the incoming
    gradient spread over each atom's orbitals (or taken per orbital), on
    every stored entry; water with ragged 4x1 / 1x4 / 1x1 blocks."""
    import torch
    from paper_1002_1202_gb300.autograd import mulliken_charges
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=True)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    Sv = torch.tensor(s.S_vals, dtype=torch.float64, device="cuda", requires_grad=True)
    Hv = torch.tensor(_block_values(s, H), dtype=torch.float64, device="cuda", requires_grad=True)
    q = mulliken_charges((s.orb_per_atom, s.brow_ptr, s.bcol), Sv, Hv, z, w, per_orbital=per_orbital)
    q_orb = dense.mulliken_orbital(H, S, z, w, 2.0)
    qd = q_orb if per_orbital else dense.mulliken_atom(q_orb, s.orbital_atom(), s.n_atoms)
    assert np.abs(q.detach().cpu().numpy() - qd).max() <= 1e-8 * np.abs(qd).max()
    u = np.random.default_rng(12).standard_normal(len(qd))
    (q * torch.tensor(u, device="cuda")).sum().backward()
    v = u if per_orbital else np.repeat(u, s.orb_per_atom)
    gHd, gSd = dense.mulliken_vjp(H, S, z, w, v)
    mask = _dense_blocks(s, np.ones(len(s.S_vals))) > 0
    gH = _dense_blocks(s, Hv.grad.cpu().numpy())
    gS = _dense_blocks(s, Sv.grad.cpu().numpy())
    assert np.abs(gH[mask] - gHd[mask]).max() <= 1e-7 * np.abs(gHd).max()
    assert np.abs(gS[mask] - gSd[mask]).max() <= 1e-7 * np.abs(gSd).max()

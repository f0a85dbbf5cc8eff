"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Plain FP64 path: true relative residual <= 1e-8 per shift, Green's function
elements within the forward-error bound cond(A) * 1e-8 of the dense solve,
Mulliken populations within 1e-6 e per orbital/atom of the dense definition.
Fixed-iteration runs are compared with the oracle's method, which runs the
same recurrences in the same order, to 1e-9 (1e-8 with forced switches).
"""
import math

import numpy as np
import pytest

from tbinputs import si_system, water_system, linspace_grid, gauss_legendre_grid, choose_columns
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


def _c1_case():
    """Si 64 atoms, sp3 (N = 256), 32 shifts on [-20, 5] eV + 0.01i, 8 columns."""
    s = si_system((2, 2, 2), sigma=0.05, seed=1, cutoff=4.0)
    z, w = linspace_grid(32)
    cols = choose_columns(256, 8, seed=2)
    return s, z, w, cols


@pytest.fixture(scope="module")
def c1():
    s, z, w, cols = _c1_case()
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    return s, H, S, z, w, cols


@pytest.fixture(scope="module")
def c1_ref(c1):
    s, H, S, z, w, cols = c1
    return dense.green_columns(H, S, z, cols)


@pytest.fixture(scope="module")
def h1(P, c1):
    return P.tb_create_system(c1[0])


@pytest.fixture(params=[0, 1, 2], ids=["fp64", "mixed", "mixed-cg"])
def prec(request):
    """TB_FP64; TB_MIXED with its default Chebyshev corrections inside FP64
    refinement; TB_MIXED with FP32 CG corrections (2 here): all must meet
    the same parity bars."""
    return request.param


def _pm(prec):
    """Options of a `prec` case."""
    return dict(precision=min(prec, 1), inner_method=1 if prec == 2 else 0)


def _true_rel_res(H, S, z, X, cols):
    out = np.zeros((len(z), len(cols)))
    for k, zk in enumerate(z):
        A = dense.shifted_matrix(H, S, zk)
        for c, j in enumerate(cols):
            b = np.zeros(S.shape[0])
            b[j] = 1.0
            out[k, c] = np.linalg.norm(b - A @ X[k, c]) / np.linalg.norm(b)
    return out


def test_full_mode_c1(P, c1, c1_ref, h1, prec):
    s, H, S, z, w, cols = c1
    x, st = P.tb_shifted_cocg(h1, z, cols, opts=P.tb_default_opts(**_pm(prec)))
    X = x.cpu().numpy()
    assert st["status"] == "TB_OK" and st["unconverged"] == 0
    assert np.all(st["conv_iter"] > 0) and st["switches"] >= 1
    res = _true_rel_res(H, S, z, X, cols)
    assert res.max() <= 1e-8, res.max()
    ref = np.transpose(c1_ref, (0, 2, 1))
    # forward error <= cond(A) * residual; cond(A) ~ ||A|| / eta ~ 1e4 here
    assert np.abs(X - ref).max() <= 1e4 * 1e-8 * np.abs(ref).max()


def test_complex_symmetry(P, c1, h1):
    s, H, S, z, w, _ = c1
    cols = [10, 11, 57]
    x, _ = P.tb_shifted_cocg(h1, z[::4], cols)
    X = x.cpu().numpy()
    for a, ca in enumerate(cols):
        for b, cb in enumerate(cols):
            assert np.abs(X[:, a, cb] - X[:, b, ca]).max() <= 1e-6 * np.abs(X).max()


@pytest.mark.parametrize("force", [0, 6])
def test_fixed_iterations_match_method_oracle(P, c1, h1, force, prec):
    s, H, S, z, w, cols = c1
    n = 30
    opts = P.tb_default_opts(max_iter=n, force_switch_every=force, **_pm(prec))
    x, st = P.tb_shifted_cocg(h1, z, cols[:3], opts=opts, allow_unconverged=True)
    X = x.cpu().numpy()
    for c, j in enumerate(cols[:3]):
        ref = method.generalized_shifted_cocg(H, S, z, int(j), max_iter=n, force_switch_every=force)["x"]
        scale = np.abs(ref).max()
        assert np.abs(X[:, c] - ref).max() <= (1e-9 if force == 0 else 1e-7) * scale


def test_green_elements(P, c1, c1_ref, h1):
    s, H, S, z, w, cols = c1
    rng = np.random.default_rng(11)
    row_ptr = [0]
    rows = []
    for j in cols:
        r = sorted(set([int(j)] + list(rng.choice(256, 5, replace=False))))
        rows += r
        row_ptr.append(len(rows))
    G, st = P.tb_green_elements(h1, z, cols, row_ptr, rows)
    G = G.cpu().numpy()
    assert st["status"] == "TB_OK"
    for c in range(len(cols)):
        for m in range(row_ptr[c], row_ptr[c + 1]):
            ref = c1_ref[:, rows[m], c]
            assert np.abs(G[m] - ref).max() <= 1e-4 * np.abs(c1_ref[:, :, c]).max()
    # projected rows equal the rows of the full solution (same recurrences)
    x, _ = P.tb_shifted_cocg(h1, z, cols)
    X = x.cpu().numpy()
    for c in range(len(cols)):
        for m in range(row_ptr[c], row_ptr[c + 1]):
            assert np.abs(G[m] - X[:, c, rows[m]]).max() <= 1e-10 * np.abs(X[:, c]).max()


@pytest.fixture(scope="module")
def c1_mulliken(c1):
    s, H, S, z, w, cols = c1
    return dense.mulliken_orbital(H, S, z, w, 2.0)


def test_mulliken_orbital(P, c1, c1_mulliken, h1, prec):
    s, H, S, z, w, cols = c1
    q, st = P.tb_mulliken_orbital(h1, z, w, cols, 2.0, opts=P.tb_default_opts(**_pm(prec)))
    q = q.cpu().numpy()
    assert np.abs(q - c1_mulliken[cols]).max() <= 1e-6


def test_mulliken_charges_and_sum_rule(P, c1, c1_mulliken, h1, prec):
    s, H, S, z, w, cols = c1
    q, st = P.tb_mulliken_charges(h1, z, w, 2.0, opts=P.tb_default_opts(**_pm(prec)))
    q = q.cpu().numpy()
    ref = dense.mulliken_atom(c1_mulliken, s.orbital_atom(), s.n_atoms)
    assert np.abs(q - ref).max() <= 1e-6
    import scipy.linalg as sl
    eig = sl.eigh(H, S, eigvals_only=True)
    assert abs(q.sum() - dense.electron_count_closed_form(eig, z, w)) <= 1e-6 * s.n_atoms


def test_host_output_buffers(P, c1, h1):
    s, H, S, z, w, cols = c1
    out = np.zeros((len(cols),))
    q_host, _ = P.tb_mulliken_orbital(h1, z, w, cols, 2.0, out=out)
    q_dev, _ = P.tb_mulliken_orbital(h1, z, w, cols, 2.0)
    assert np.array_equal(q_host, q_dev.cpu().numpy())


def test_explicit_H_same_as_ased(P, c1, h1):
    s, H, S, z, w, cols = c1
    # block values of the oracle's ASED H in the input layout
    oo = s.orb_offset()
    bo = s.block_offsets()
    hv = np.zeros_like(s.S_vals)
    for i in range(s.n_atoms):
        for b in range(s.brow_ptr[i], s.brow_ptr[i + 1]):
            j = s.bcol[b]
            hv[bo[b]:bo[b + 1]] = H[oo[i]:oo[i] + 4, oo[j]:oo[j] + 4].ravel()
    h2 = P.tb_create_system(s, explicit_H=hv)
    x1, _ = P.tb_shifted_cocg(h1, z[:8], cols[:2])
    x2, _ = P.tb_shifted_cocg(h2, z[:8], cols[:2])
    assert np.abs(x1.cpu().numpy() - x2.cpu().numpy()).max() <= 1e-12 * np.abs(x1.cpu().numpy()).max()


def test_non_identity_diagonal_blocks(P, c1, prec):
    """Orbitals rescaled by a seeded diagonal D (S' = D S D, H' = D H D):
    the diagonal blocks of S' are no longer the identity, so every product
    keeps them (the path that skips identity diagonal blocks is not taken);
    the solutions meet the same true-residual bar and the populations the
    same 1e-6 e bar against the dense definitions of the rescaled system."""
    s, H, S, z, w, cols = c1
    d = np.random.default_rng(11).uniform(0.8, 1.25, S.shape[0])
    S2, H2 = S * np.outer(d, d), H * np.outer(d, d)
    oo, bo = s.orb_offset(), s.block_offsets()
    sv, hv = np.zeros_like(s.S_vals), np.zeros_like(s.S_vals)
    for i in range(s.n_atoms):
        for b in range(s.brow_ptr[i], s.brow_ptr[i + 1]):
            j = s.bcol[b]
            sv[bo[b]:bo[b + 1]] = S2[oo[i]:oo[i] + 4, oo[j]:oo[j] + 4].ravel()
            hv[bo[b]:bo[b + 1]] = H2[oo[i]:oo[i] + 4, oo[j]:oo[j] + 4].ravel()
    h = P.tb_create(s.orb_per_atom, s.brow_ptr, s.bcol, sv, hv, None, s.K)
    zz = z[::4]
    x, _ = P.tb_shifted_cocg(h, zz, cols[:4], opts=P.tb_default_opts(**_pm(prec)))
    assert _true_rel_res(H2, S2, zz, x.cpu().numpy(), cols[:4]).max() <= 1e-8
    q, _ = P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=P.tb_default_opts(**_pm(prec)))
    assert np.abs(q.cpu().numpy() - dense.mulliken_orbital(H2, S2, z, w, 2.0)[cols]).max() <= 1e-6


def test_panel_split_with_ragged_tail(P, c1, c1_ref, h1, prec):
    s, H, S, z, w, cols = c1
    cols13 = choose_columns(256, 13, seed=7)
    zz = z[::6]
    opts = P.tb_default_opts(panel=8, **_pm(prec))
    x, st = P.tb_shifted_cocg(h1, zz, cols13, opts=opts)
    X = x.cpu().numpy()
    res = _true_rel_res(H, S, zz, X, cols13)
    assert res.max() <= 1e-8


def test_single_shift_single_column(P, c1, h1):
    s, H, S, z, w, cols = c1
    x, st = P.tb_shifted_cocg(h1, [z[5]], [int(cols[0])])
    X = x.cpu().numpy()
    assert _true_rel_res(H, S, [z[5]], X, [cols[0]]).max() <= 1e-8
    assert st["switches"] == 0


def test_water_ragged_blocks(P, prec):
    s = water_system(32, seed=4)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    z, w = linspace_grid(8, -35.0, 5.0, 0.05)
    cols = [0, 1, 4, s.n_orb - 1]
    h = P.tb_create_system(s)
    opts = P.tb_default_opts(**_pm(prec))
    x, st = P.tb_shifted_cocg(h, z, cols, opts=opts)
    X = x.cpu().numpy()
    assert _true_rel_res(H, S, z, X, cols).max() <= 1e-8
    q, _ = P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=opts)
    ref = dense.mulliken_orbital(H, S, z, w, 2.0)[cols]
    assert np.abs(q.cpu().numpy() - ref).max() <= 1e-6


def test_lanczos(P, c1, h1):
    s, H, S, z, w, cols = c1
    j = 9
    a, b, nrm = P.tb_generalized_lanczos(h1, j, 100)
    ar, br, nr = method.generalized_lanczos(H, S, j, 100)
    assert abs(nrm - nr) <= 1e-12 * nr
    assert np.abs(a[:20] - ar[:20]).max() <= 1e-8 * np.abs(ar).max()
    assert np.abs(b[:21] - br[:21]).max() <= 1e-8 * np.abs(br).max()
    zz = np.array([-5.0 + 2.0j, 2.0 + 2.0j])
    g = method.lanczos_green(a, b, nrm, zz)
    ref = dense.green_columns(H, S, zz, [j])[:, j, 0]
    assert np.abs(g - ref).max() <= 1e-8 * np.abs(ref).max()
    # the continued fraction on the device: the oracle's on the same
    # coefficients, and the dense G_jj (local density of states)
    zl = np.linspace(-25.0, 10.0, 301) + 2.0j
    gd = P.tb_lanczos_green(a, b, nrm, zl)
    go = method.lanczos_green(a, b, nrm, zl)
    assert np.abs(gd - go).max() <= 1e-12 * np.abs(go).max()
    gref = dense.green_columns(H, S, zl[::30], [j])[:, j, 0]
    assert np.abs(gd[::30] - gref).max() <= 1e-8 * np.abs(gref).max()
    with pytest.raises(P.TBError):
        P.tb_lanczos_green(a, b, float("nan"), zl)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_lanczos_batch(P, c1, h1, prec):
    """Lanczos processes of several columns in one panel (two panels with a
    ragged tail at panel 4) against the oracle's process per column; the
    single-column call is the batch of one."""
    s, H, S, z, w, cols = c1
    js = [9, 0, 255, 100, 31, 64]
    a, b, nrm = P.tb_generalized_lanczos_batch(h1, js, 60, opts=P.tb_default_opts(precision=prec, panel=4,
                                                                                   inner_tol=1e-13))
    for c, j in enumerate(js):
        ar, br, nr = method.generalized_lanczos(H, S, j, 60)
        assert abs(nrm[c] - nr) <= 1e-12 * nr
        assert np.abs(a[c, :20] - ar[:20]).max() <= 1e-8 * np.abs(ar).max()
        assert np.abs(b[c, :21] - br[:21]).max() <= 1e-8 * np.abs(br).max()
    # continued fractions of all processes at once (local densities of states)
    zl = np.linspace(-25.0, 10.0, 41) + 2.0j
    Gb = P.tb_lanczos_green_batch(a, b, nrm, zl)
    for c in range(len(js)):
        go = method.lanczos_green(a[c], b[c], nrm[c], zl)
        assert np.abs(Gb[c] - go).max() <= 1e-12 * np.abs(go).max()
    if prec == 0:
        # same process, other panel width (other reduction order): Lanczos
        # amplifies rounding once orthogonality is lost, so compare early steps
        a1, b1, n1 = P.tb_generalized_lanczos(h1, js[3], 60)
        assert np.abs(a1[:20] - a[3, :20]).max() <= 1e-10 * np.abs(a1).max()
        assert abs(n1 - nrm[3]) <= 1e-13 * n1


def test_not_converged_status(P, c1, h1):
    s, H, S, z, w, cols = c1
    opts = P.tb_default_opts(max_iter=5)
    with pytest.raises(P.TBError) as e:
        P.tb_shifted_cocg(h1, z, cols[:2], opts=opts)
    assert e.value.status == 6
    x, st = P.tb_shifted_cocg(h1, z, cols[:2], opts=opts, allow_unconverged=True)
    assert st["unconverged"] == 2 * 32


def test_invalid_arguments(P, c1, h1):
    s, H, S, z, w, cols = c1
    for bad in ([-1], [256], []):
        with pytest.raises(P.TBError) as e:
            P.tb_shifted_cocg(h1, z[:2], bad)
        assert e.value.status == 1
    with pytest.raises(P.TBError):
        P.tb_shifted_cocg(h1, z[:2], [0], opts=P.tb_default_opts(seed=5))
    with pytest.raises(P.TBError):
        P.tb_shifted_cocg(h1, z[:2], [0], opts=P.tb_default_opts(panel=48))


def test_overlap_not_positive_definite(P, c1, prec):
    s = c1[0]
    sv = s.S_vals.copy()
    bo = s.block_offsets()
    for i in range(s.n_atoms):
        for b in range(s.brow_ptr[i], s.brow_ptr[i + 1]):
            if s.bcol[b] != i:
                sv[bo[b]:bo[b + 1]] *= 3.0       # eigenvalues 1 + 3(l - 1) < 0
    h = P.tb_create(s.orb_per_atom, s.brow_ptr, s.bcol, sv, None, s.eps, s.K)
    with pytest.raises(P.TBError) as e:
        P.tb_shifted_cocg(h, linspace_grid(4)[0], [0], opts=P.tb_default_opts(**_pm(prec)))
    assert e.value.status == 3


def test_max_shift_count(P, c1, h1):
    s, H, S, z, w, cols = c1
    zz = np.linspace(-20, 5, 1024) + 0.05j
    opts = P.tb_default_opts(tol=1e-9)
    G, st = P.tb_green_elements(h1, zz, [int(cols[0])], [0, 1], [int(cols[0])], opts=opts)
    ref = dense.green_columns(H, S, zz[::97], [int(cols[0])])[:, cols[0], 0]
    assert np.abs(G.cpu().numpy()[0, ::97] - ref).max() <= 1e-4 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# full-size workload (Si 4096 atoms, N = 16384, 256 Gauss-Legendre shifts),
# bench launch configuration (panel of 64 columns, Mulliken projection):
# sampled columns against the oracle's method after the same number of steps
# ---------------------------------------------------------------------------
@pytest.mark.slow
@pytest.mark.parametrize("precision,ncols,panel,sample,rtol",
                         [(0, 64, 64, (0, 37), 1e-9), (1, 1024, 256, (0, 300, 700, 1023), 1e-7)],
                         ids=["fp64", "mixed-bench-launch"])
def test_full_size_sampled_columns(P, precision, ncols, panel, sample, rtol):
    """The benchmark's system and shifts (Si 4096 atoms, 256 Gauss-Legendre
    shifts at 0.01 eV); the mixed case in the benchmark's launch
    configuration (1024 columns as four panels of 256 in flight, tol 1e-8,
    inner 1e-12).  Sampled columns, from every panel, after 12 outer steps,
    against the oracle's method on the same column.  Both sides solve
    S r' = r only to inner_tol = 1e-12, by different solvers (FP64 CG against
    FP32 corrections inside FP64 refinement); to first order the populations then
    differ by up to n cond(A) inner_tol ~ 12 x (40 eV / 0.01 eV) x 1e-12
    ~ 5e-8, hence 1e-7 for the mixed case (the FP64 case runs the oracle's
    own CG steps and agrees to 1e-9).  The mixed case runs the default
    Chebyshev corrections inside FP64 refinement."""
    s = si_system((8, 8, 8), sigma=0.05, seed=3, cutoff=4.0)
    z, w = gauss_legendre_grid(256, -20.0, 5.0, 0.01)
    cols = choose_columns(s.n_orb, ncols, seed=5)
    n = 12
    h = P.tb_create_system(s)
    opts = P.tb_default_opts(max_iter=n, panel=panel, precision=precision, tol=1e-8, inner_tol=1e-12)
    q, st = P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=opts, allow_unconverged=True)
    q = q.cpu().numpy()
    Sc = s.to_csr()
    Hc = dense.ased_hamiltonian_sparse(Sc, s.eps, s.K, s.orbital_atom())
    for c in sample:
        j = int(cols[c])
        F = Sc[j].toarray()
        out = method.generalized_shifted_cocg(Hc, Sc, z, j, max_iter=n, keep_full=False, functionals=F,
                                              tol=1e-8, inner_tol=1e-12)
        qref = -(2.0 / math.pi) * np.imag(np.sum(w * out["t"][:, 0]))
        assert abs(q[c] - qref) <= rtol * max(1.0, abs(qref))


@pytest.mark.slow
def test_full_size_columns_to_solution(P):
    """Columns of the benchmark's system (Si 4096 atoms, 256 Gauss-Legendre
    shifts at 0.01 eV) run to the 1e-8 residual, mixed precision: every shift
    of every column converges, and the true residual of the solutions at a
    sample of shifts spread over the window -- the largest Krylov counts
    included -- computed on the CPU from the oracle's sparse H and S, is
    within 1e-8 x 10 (the recursive residual drifts from the true one by
    the inexact inner solves, ~ n cond(A) inner_tol)."""
    s = si_system((8, 8, 8), sigma=0.05, seed=3, cutoff=4.0)
    z, _ = gauss_legendre_grid(256, -20.0, 5.0, 0.01)
    cols = choose_columns(s.n_orb, 2, seed=9)
    ks = np.array([0, 40, 90, 128, 170, 215, 255])
    h = P.tb_create_system(s)
    opts = P.tb_default_opts(max_iter=100000, precision=1, tol=1e-8, inner_tol=1e-12)
    x, st = P.tb_shifted_cocg(h, z[ks], cols, opts=opts)
    assert st["status"] == "TB_OK"
    X = x.cpu().numpy()
    Sc = s.to_csr()
    Hc = dense.ased_hamiltonian_sparse(Sc, s.eps, s.K, s.orbital_atom())
    worst = 0.0
    for a, k in enumerate(ks):
        A = z[k] * Sc - Hc
        for c, j in enumerate(cols):
            b = np.zeros(s.n_orb)
            b[j] = 1.0
            worst = max(worst, np.linalg.norm(b - A @ X[a, c]))
    assert worst <= 1e-7, worst


def test_mixed_inner_tolerances(P, c1, h1):
    """TB_MIXED with a looser outer inner_tol still meets the residual bar,
    and invalid FP32 round tolerances are rejected."""
    s, H, S, z, w, cols = c1
    opts = P.tb_default_opts(precision=1, inner_tol=1e-12, inner_lo_tol=1e-5)
    x, st = P.tb_shifted_cocg(h1, z[::4], cols[:3], opts=opts)
    assert _true_rel_res(H, S, z[::4], x.cpu().numpy(), cols[:3]).max() <= 1e-8
    for bad in (0.0, 1.0, -1e-6):
        with pytest.raises(P.TBError):
            P.tb_shifted_cocg(h1, z[:2], [0], opts=P.tb_default_opts(precision=1, inner_lo_tol=bad))
    with pytest.raises(P.TBError):
        P.tb_shifted_cocg(h1, z[:2], [0], opts=P.tb_default_opts(precision=2))


@pytest.mark.parametrize("group", ["0", "2", "16"], ids=["gather", "group2", "group16"])
def test_mixed_spmv_forms(P, c1, monkeypatch, group):
    """The FP32 CG SpMV of TB_MIXED in its register-gather form (no atom
    groups) and its grouped shared-memory form (groups of 2 and 16 atoms,
    40 columns: a 64-column panel, two 32-column slices, ragged tail) give
    the oracle's fixed-iteration iterates and fully converged solutions."""
    s, H, S, z, w, cols = c1
    monkeypatch.setenv("TB_SPMV_GROUP", group)
    h = P.tb_create_system(s)
    monkeypatch.delenv("TB_SPMV_GROUP")
    many = choose_columns(256, 40, seed=5)
    n = 25
    opts = P.tb_default_opts(max_iter=n, precision=1, inner_method=1)
    x, st = P.tb_shifted_cocg(h, z[::4], many, opts=opts, allow_unconverged=True)
    X = x.cpu().numpy()
    for c in (0, 17, 39):
        ref = method.generalized_shifted_cocg(H, S, z[::4], int(many[c]), max_iter=n)["x"]
        assert np.abs(X[:, c] - ref).max() <= 1e-9 * np.abs(ref).max()
    x, st = P.tb_shifted_cocg(h, z[::4], many, opts=P.tb_default_opts(precision=1, inner_method=1))
    assert st["status"] == "TB_OK"
    assert _true_rel_res(H, S, z[::4], x.cpu().numpy(), many).max() <= 1e-8


def test_mixed_spmv_grouped_water(P, monkeypatch):
    """Grouped FP32 CG SpMV on ragged blocks (O: 4 orbitals, H: 1) with a
    partial last group: converged Mulliken populations of 36 columns."""
    s = water_system(32, seed=4)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    z, w = linspace_grid(8, -35.0, 5.0, 0.05)
    cols = list(range(0, s.n_orb, max(1, s.n_orb // 36)))[:36]
    monkeypatch.setenv("TB_SPMV_GROUP", "16")
    h = P.tb_create_system(s)
    monkeypatch.delenv("TB_SPMV_GROUP")
    q, st = P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=P.tb_default_opts(precision=1, inner_method=1))
    ref = dense.mulliken_orbital(H, S, z, w, 2.0)[cols]
    assert np.abs(q.cpu().numpy() - ref).max() <= 1e-6


@pytest.mark.parametrize("which", ["si64", "water8"])
def test_overlap_bounds(P, c1, which):
    """The Chebyshev bounds enclose the spectrum of S (dense eigenvalues)
    and are tight to within their margins."""
    if which == "si64":
        s = c1[0]
    else:
        s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    ev = np.linalg.eigvalsh(s.dense_S())
    lo, hi = P.tb_overlap_bounds(P.tb_create_system(s))
    assert 0.0 < lo <= ev[0] and hi >= ev[-1]
    assert lo >= 0.9 * ev[0] and hi <= 1.05 * ev[-1]


def test_chebyshev_and_cg_corrections_agree(P, c1, h1):
    """Mixed precision with Chebyshev and with CG corrections: converged
    Mulliken populations of the same columns agree with each other and the
    oracle to 1e-7 e; the Chebyshev solve launches fewer inner steps per
    refinement round than CG needs iterations plus its scalar tails."""
    s, H, S, z, w, cols = c1
    ref = dense.mulliken_orbital(H, S, z, w, 2.0)[cols]
    qs = []
    for m in (0, 1):
        q, st = P.tb_mulliken_orbital(h1, z, w, cols, 2.0, opts=P.tb_default_opts(precision=1, inner_method=m))
        assert st["status"] == "TB_OK"
        qs.append(q.cpu().numpy())
        assert np.abs(qs[-1] - ref).max() <= 1e-7
    assert np.abs(qs[0] - qs[1]).max() <= 1e-7


def test_graph_and_direct_launches_agree(P, c1, h1, tmp_path):
    """The Chebyshev steps of a round replayed as a CUDA graph (default) and
    launched one by one (TB_GRAPHS=0, in a child process) give bit-identical
    populations: the same kernels with the same arguments in the same
    order."""
    import os
    import subprocess
    import sys
    s, H, S, z, w, cols = c1
    q, st = P.tb_mulliken_orbital(h1, z, w, cols, 2.0, opts=P.tb_default_opts(precision=1, max_iter=30),
                                  allow_unconverged=True)
    out = tmp_path / "q.npy"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = (
        "import numpy as np, paper_1002_1202_gb300 as P\n"
        "from tests.test_gpu_parity import _c1_case\n"
        "s, z, w, cols = _c1_case()\n"
        "h = P.tb_create_system(s)\n"
        "q, st = P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=P.tb_default_opts(precision=1, max_iter=30),"
        " allow_unconverged=True)\n"
        f"np.save({str(out)!r}, q.cpu().numpy())\n")
    env = dict(os.environ, TB_GRAPHS="0", PYTHONPATH=root)
    subprocess.run([sys.executable, "-c", child], env=env, cwd=root, check=True, timeout=600)
    assert np.array_equal(np.load(out), q.cpu().numpy())

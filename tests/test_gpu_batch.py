"""Ragged batches (block-diagonal handle of independent systems) on the GPU:
a batch solve gives the per-system solves, columns of different systems
share panels, and nothing leaks across systems."""
import numpy as np
import pytest

from tbinputs import water_system, si_system, gauss_legendre_grid
from oracle import dense

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
def systems():
    return [water_system(8, seed=4, cutoff=3.0, excess_proton=False),
            si_system((2, 2, 2), sigma=0.05, seed=1),
            water_system(16, seed=7, cutoff=3.0)]


@pytest.fixture(scope="module")
def grid():
    return gauss_legendre_grid(32, -40.0, 0.0, 1.0)


def test_batch_offsets(P, systems):
    h = P.tb_create_batch(systems)
    assert list(h.atom_off) == list(np.cumsum([0] + [s.n_atoms for s in systems]))
    assert list(h.orb_off) == list(np.cumsum([0] + [s.n_orb for s in systems]))
    assert h.n_orb == sum(s.n_orb for s in systems)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_batch_charges_equal_per_system(P, systems, grid, prec):
    z, w = grid
    opts = P.tb_default_opts(precision=prec)
    hb = P.tb_create_batch(systems)
    qb, st = P.tb_mulliken_charges(hb, z, w, opts=opts)
    qb = qb.cpu().numpy()
    for i, s in enumerate(systems):
        q, _ = P.tb_mulliken_charges(P.tb_create_system(s), z, w, opts=opts)
        assert np.abs(qb[hb.atom_off[i]:hb.atom_off[i + 1]] - q.cpu().numpy()).max() <= 1e-9
    # one system against the dense definition
    s = systems[0]
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    ref = dense.mulliken_atom(dense.mulliken_orbital(H, S, z, w), s.orbital_atom(), s.n_atoms)
    assert np.abs(qb[:s.n_atoms] - ref).max() <= 1e-8


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_batch_columns_stay_in_their_system(P, systems, grid, prec):
    z, w = grid
    z = z[::4]
    hb = P.tb_create_batch(systems)
    picks = [(0, 3), (1, 0), (1, 200), (2, 5), (0, 40)]
    cols = [int(hb.orb_off[i] + j) for i, j in picks]
    opts = P.tb_default_opts(precision=prec)
    x, st = P.tb_shifted_cocg(hb, z, cols, opts=opts)
    X = x.cpu().numpy()
    for c, (i, j) in enumerate(picks):
        lo, hi = hb.orb_off[i], hb.orb_off[i + 1]
        outside = np.concatenate([X[:, c, :lo], X[:, c, hi:]], axis=1)
        assert np.all(outside == 0)
        xs, _ = P.tb_shifted_cocg(P.tb_create_system(systems[i]), z, [j], opts=opts)
        ref = xs.cpu().numpy()[:, 0]
        assert np.abs(X[:, c, lo:hi] - ref).max() <= 1e-9 * np.abs(ref).max()


def test_batch_green_elements_and_stats(P, systems, grid):
    z, w = grid
    z = z[::4]
    hb = P.tb_create_batch(systems)
    o1 = int(hb.orb_off[1])
    cols = [2, o1 + 7, o1 + 100]
    # rows of the column's own system and of another system (those are zero)
    rows_per_col = [[2, 5, o1 + 3], [o1 + 7, o1 + 9, 4], [o1 + 100, int(hb.orb_off[2]) + 1]]
    row_ptr = np.cumsum([0] + [len(r) for r in rows_per_col])
    rows = [r for rr in rows_per_col for r in rr]
    G, st = P.tb_green_elements(hb, z, cols, row_ptr, rows)
    G = G.cpu().numpy()
    x, st2 = P.tb_shifted_cocg(hb, z, cols)
    X = x.cpu().numpy()
    for c in range(len(cols)):
        for m in range(row_ptr[c], row_ptr[c + 1]):
            r = rows[m]
            same = np.searchsorted(hb.orb_off, r, side="right") == np.searchsorted(hb.orb_off, cols[c], side="right")
            if same:
                assert np.abs(G[m] - X[:, c, r]).max() <= 1e-10 * np.abs(X[:, c]).max()
            else:
                assert np.all(G[m] == 0)
    assert st["outer_iterations"] > 0 and st["status"] == "TB_OK"
    # per-(column, shift) convergence steps come back in the caller's column order
    conv = np.asarray(st2["conv_iter"]).reshape(len(cols), len(z))
    assert np.all(conv >= 0)
    for c, j in enumerate(cols):
        sys = int(np.searchsorted(hb.orb_off, j, side="right")) - 1
        _, sts = P.tb_shifted_cocg(P.tb_create_system(systems[sys]), z, [j - int(hb.orb_off[sys])])
        # same recurrences; rounding order differs with the panel width (+-1 step)
        assert np.abs(conv[c] - np.asarray(sts["conv_iter"]).reshape(1, len(z))[0]).max() <= 1


def _batch_case():
    systems = [water_system(8, seed=4, cutoff=3.0, excess_proton=False),
               si_system((2, 2, 2), sigma=0.05, seed=1),
               water_system(16, seed=7, cutoff=3.0)]
    z, w = gauss_legendre_grid(32, -40.0, 0.0, 1.0)
    return systems, z, w


def test_step_graphs_on_a_ragged_batch(P, tmp_path):
    """Mixed path on a ragged batch (water with 4x1 / 1x1 blocks, silicon):
    outer steps replayed as one CUDA graph per panel (default) and launched
    one by one (TB_STEP_GRAPHS=0, in a child process) give bit-identical
    populations -- the same kernels with the same arguments in the same
    order -- and both equal the dense definition on the first system."""
    import os
    import subprocess
    import sys
    systems, z, w = _batch_case()
    hb = P.tb_create_batch(systems)
    q, st = P.tb_mulliken_charges(hb, z, w, opts=P.tb_default_opts(precision=1))
    assert st["status"] == "TB_OK"
    q = q.cpu().numpy()
    s = systems[0]
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    ref = dense.mulliken_atom(dense.mulliken_orbital(H, S, z, w), s.orbital_atom(), s.n_atoms)
    assert np.abs(q[:s.n_atoms] - ref).max() <= 1e-8
    out = tmp_path / "q.npy"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = (
        "import numpy as np, paper_1002_1202_gb300 as P\n"
        "from tests.test_gpu_batch import _batch_case\n"
        "systems, z, w = _batch_case()\n"
        "hb = P.tb_create_batch(systems)\n"
        "q, st = P.tb_mulliken_charges(hb, z, w, opts=P.tb_default_opts(precision=1))\n"
        f"np.save({str(out)!r}, q.cpu().numpy())\n")
    env = dict(os.environ, TB_STEP_GRAPHS="0", PYTHONPATH=root)
    subprocess.run([sys.executable, "-c", child], env=env, cwd=root, check=True, timeout=600)
    assert np.array_equal(np.load(out), q)


def test_autotune_choice_is_used(P):
    """tb_autotune times the launch candidates on the handle's own system,
    orders them by rate and keeps the best for its size class; a later call
    with panel 0 then runs with it and gives the populations of an explicit
    call with the same choice."""
    s = si_system((4, 4, 2), sigma=0.05, seed=1)
    z, w = gauss_legendre_grid(32, -20.0, 5.0, 1.0)
    h = P.tb_create_system(s)
    base = P.tb_default_opts(precision=1)
    cands = P.tb_autotune(h, z, w, opts=base, iters=2)
    rates = [c["rate"] for c in cands]
    assert len(cands) >= 8 and rates == sorted(rates, reverse=True) and rates[-1] > 0
    assert {c["ctas_per_sm"] for c in cands} == {3, 4}
    best = cands[0]
    cols = np.arange(0, s.n_orb, 5, dtype=np.int32)
    q_auto, st = P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=P.tb_default_opts(precision=1, panel=0))
    assert st["status"] == "TB_OK"
    q_ref, _ = P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=P.tb_default_opts(precision=1, panel=best["panel"]))
    assert np.abs(q_auto.cpu().numpy() - q_ref.cpu().numpy()).max() <= 1e-9


def test_ragged_chebyshev_step_equals_padded(P, tmp_path):
    """Water (O: s, p; H: s) with exact orbital counts in the Chebyshev step
    (compact blocks, one gathered row per H neighbour, one output row per H
    atom) and in the double-float SpMVs (default) against the padded forms
    (TB_CHEB_RAG=0, TB_DF_RAG=0, child process): the padded forms only add
    exact zeros (padded rows of the vectors) in the same order, so the
    populations are bit-identical, on one box and on a ragged batch."""
    import os
    import subprocess
    import sys
    systems, z, w = _batch_case()
    hb = P.tb_create_batch(systems)
    q, st = P.tb_mulliken_charges(hb, z, w, opts=P.tb_default_opts(precision=1))
    assert st["status"] == "TB_OK"
    h1 = P.tb_create_system(systems[2])
    q1, _ = P.tb_mulliken_charges(h1, z, w, opts=P.tb_default_opts(precision=1))
    out = tmp_path / "q.npz"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = (
        "import numpy as np, paper_1002_1202_gb300 as P\n"
        "from tests.test_gpu_batch import _batch_case\n"
        "systems, z, w = _batch_case()\n"
        "hb = P.tb_create_batch(systems)\n"
        "q, st = P.tb_mulliken_charges(hb, z, w, opts=P.tb_default_opts(precision=1))\n"
        "h1 = P.tb_create_system(systems[2])\n"
        "q1, _ = P.tb_mulliken_charges(h1, z, w, opts=P.tb_default_opts(precision=1))\n"
        f"np.savez({str(out)!r}, q=q.cpu().numpy(), q1=q1.cpu().numpy())\n")
    env = dict(os.environ, TB_CHEB_RAG="0", TB_DF_RAG="0", PYTHONPATH=root)
    subprocess.run([sys.executable, "-c", child], env=env, cwd=root, check=True, timeout=600)
    ref = np.load(out)
    assert np.array_equal(ref["q"], q.cpu().numpy())
    assert np.array_equal(ref["q1"], q1.cpu().numpy())

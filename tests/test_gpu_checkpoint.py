"""Energy-point checkpointing (tb_solve_opts.state_bytes): with a state
budget too small for all shifts at once, the shifts are solved in chunks,
each a separate shifted COCG whose seed sequence is recomputed, and each
chunk's full solutions go to the caller's output -- device or host memory --
before the next chunk starts.  Every shift's solution is unique (Im z != 0),
so the chunked call must give the solutions of one call to within the
solver's tolerance, and each must meet the true-residual bar against the
dense operator; the Mulliken vector-Jacobian product, summed over the
shifts chunk by chunk, must equal the unchunked one."""
import numpy as np
import pytest

from tbinputs import si_system, water_system, linspace_grid
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
def si():
    s = si_system((2, 2, 2), sigma=0.05, seed=1)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    return s, H, S


def _true_residuals(H, S, z, cols, X):
    N = S.shape[0]
    worst = 0.0
    for k, zk in enumerate(z):
        A = dense.shifted_matrix(H, S, zk)
        for c, j in enumerate(cols):
            b = np.zeros(N)
            b[j] = 1.0
            worst = max(worst, np.linalg.norm(b - A @ X[k, c]))
    return worst


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("where", ["device", "host"])
def test_shift_chunks_equal_one_call(P, si, prec, where):
    s, H, S = si
    z, _ = linspace_grid(16, -20.0, 5.0, 0.5)
    cols = [3, 77, 130, 201]
    h = P.tb_create_system(s)
    ref, st0 = P.tb_shifted_cocg(h, z, cols, opts=P.tb_default_opts(precision=prec))
    ref = ref.cpu().numpy()
    # per shift: x^k, p^k of one panel of 4 columns (32 B x 256 padded rows
    # x 4), plus for host outputs the chunk's device copy (16 B x 4 x 256):
    # a budget of 5 shifts' worth gives chunks of 5 (device) or 3 (host)
    per = 32 * 256 * 4
    budget = 5 * per
    opts = P.tb_default_opts(precision=prec, state_bytes=budget)
    if where == "host":
        out = np.zeros((len(z), len(cols), s.n_orb), dtype=np.complex128)
        X, st = P.tb_shifted_cocg(h, z, cols, opts=opts, out=out)
    else:
        X, st = P.tb_shifted_cocg(h, z, cols, opts=opts)
        X = X.cpu().numpy()
    assert st["status"] == "TB_OK"
    assert np.abs(X - ref).max() <= 1e-7 * np.abs(ref).max()
    assert _true_residuals(H, S, z, cols, X) <= 1e-8
    # every (column, shift) reports its convergence step from its own chunk
    assert np.all(np.asarray(st["conv_iter"]) >= 0)


def test_shift_chunks_keep_the_chosen_seed(P, si):
    """opts.seed inside a later chunk is that chunk's seed; the others start
    from their first shift.  Results as one call."""
    s, H, S = si
    z, _ = linspace_grid(12, -20.0, 5.0, 0.5)
    cols = [5, 140]
    h = P.tb_create_system(s)
    ref, _ = P.tb_shifted_cocg(h, z, cols, opts=P.tb_default_opts(seed=9))
    X, st = P.tb_shifted_cocg(h, z, cols, opts=P.tb_default_opts(seed=9, state_bytes=4 * 32 * 256 * 2))
    assert st["status"] == "TB_OK"
    assert np.abs(X.cpu().numpy() - ref.cpu().numpy()).max() <= 1e-7 * np.abs(ref.cpu().numpy()).max()


def test_mulliken_vjp_shift_chunks(P):
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    z, w = linspace_grid(16, -40.0, -8.0, 1.0)
    rng = np.random.default_rng(8)
    v = np.zeros(s.n_orb)
    v[rng.choice(s.n_orb, 8, replace=False)] = rng.standard_normal(8)
    h = P.tb_create_system(s)
    gH0, gS0, _ = P.tb_mulliken_vjp(h, z, w, v, len(s.S_vals))
    # 64 N bytes per (column, shift): a budget of 3 of them gives one column
    # and 3 shifts per chunk
    gH, gS, st = P.tb_mulliken_vjp(h, z, w, v, len(s.S_vals),
                                   opts=P.tb_default_opts(state_bytes=3 * 64 * s.n_orb))
    assert st["status"] == "TB_OK"
    assert np.abs(gH - gH0).max() <= 1e-8 * np.abs(gH0).max()
    assert np.abs(gS - gS0).max() <= 1e-8 * np.abs(gS0).max()

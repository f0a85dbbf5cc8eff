"""Charge self-consistency on the GPU (Eq. Hap-CSC) against the oracle.

The Hamiltonian update is checked through the populations it produces
(dense oracle on H0 + H^CSC), the loop against the oracle's linear-mixing
loop on the same inputs: same iteration count (+-1 at the stopping test)
and the same self-consistent charges.  The energy grid has a broadening
(2 eV) larger than its node spacing, so the populations are smooth in the
potential and the loop contracts.
"""
import numpy as np
import pytest

from tbinputs import water_system, klopman_ohno_gamma, valence_populations, gauss_legendre_grid
from oracle import dense, csc

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
def w8():
    s = water_system(8, seed=4, cutoff=3.0, excess_proton=False)
    S = s.dense_S()
    oa = s.orbital_atom()
    H0 = dense.ased_hamiltonian(S, s.eps, s.K, oa)
    gamma = 0.25 * klopman_ohno_gamma(s)
    q_ref = valence_populations(s)
    z, w = gauss_legendre_grid(128, -60.0, -8.0, 2.0)
    return s, S, oa, H0, gamma, q_ref, z, w


@pytest.fixture(scope="module")
def w8_loop(w8):
    s, S, oa, H0, gamma, q_ref, z, w = w8
    return csc.csc_loop(H0, S, oa, s.n_atoms, gamma, q_ref, z, w, mix=0.5, tol=1e-8, max_iter=60)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_csc_hamiltonian_populations(P, w8, prec):
    s, S, oa, H0, gamma, q_ref, z, w = w8
    dq = np.random.default_rng(9).standard_normal(s.n_atoms) * 0.3
    h = P.tb_create_system(s)
    P.tb_csc_hamiltonian(h, gamma, dq)
    q, st = P.tb_mulliken_charges(h, z, w, opts=P.tb_default_opts(precision=prec))
    ref = dense.mulliken_atom(dense.mulliken_orbital(csc.csc_hamiltonian(H0, S, oa, gamma, dq), S, z, w),
                              oa, s.n_atoms)
    assert np.abs(q.cpu().numpy() - ref).max() <= 1e-8
    # back to H0: the same populations as a fresh handle, bit for bit
    P.tb_csc_hamiltonian(h, None, None)
    q0, _ = P.tb_mulliken_charges(h, z, w, opts=P.tb_default_opts(precision=prec))
    q1, _ = P.tb_mulliken_charges(P.tb_create_system(s), z, w, opts=P.tb_default_opts(precision=prec))
    assert np.array_equal(q0.cpu().numpy(), q1.cpu().numpy())


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_csc_loop_matches_oracle(P, w8, w8_loop, prec):
    s, S, oa, H0, gamma, q_ref, z, w = w8
    h = P.tb_create_system(s)
    copts = P.tb_default_csc_opts(mix=0.5, scf_tol=1e-8, max_scf=60)
    q, dq, st = P.tb_csc_loop(h, z, w, gamma, q_ref, copts=copts, opts=P.tb_default_opts(precision=prec))
    assert st["status"] == "TB_OK" and st["residual"] <= 1e-8
    assert abs(st["iterations"] - w8_loop["iterations"]) <= 1
    assert np.abs(dq.cpu().numpy() - w8_loop["dq"]).max() <= 1e-7
    assert np.abs(q.cpu().numpy() - w8_loop["q"]).max() <= 1e-7
    # the handle is left at H0 + H^CSC(dq): its populations are the loop's
    q2, _ = P.tb_mulliken_charges(h, z, w, opts=P.tb_default_opts(precision=prec))
    assert np.abs(q2.cpu().numpy() - q.cpu().numpy()).max() <= 1e-9


def test_csc_loop_host_buffers_and_cap(P, w8):
    s, S, oa, H0, gamma, q_ref, z, w = w8
    h = P.tb_create_system(s)
    q_out = np.zeros(s.n_atoms)
    dq_out = np.zeros(s.n_atoms)
    dq0 = np.full(s.n_atoms, 0.01)
    copts = P.tb_default_csc_opts(mix=0.5, scf_tol=1e-8, max_scf=3)
    q, dq, st = P.tb_csc_loop(h, z, w, gamma, q_ref, dq_init=dq0, copts=copts, q_out=q_out, dq_out=dq_out,
                              allow_unconverged=True)
    assert st["status"] == "TB_ERR_NOT_CONVERGED" and st["iterations"] == 3
    ref = csc.csc_loop(H0, S, oa, s.n_atoms, gamma, q_ref, z, w, mix=0.5, tol=1e-8, max_iter=3, dq_init=dq0)
    assert not ref["converged"]
    assert np.abs(dq_out - ref["dq"]).max() <= 1e-9
    assert np.abs(q_out - ref["q"]).max() <= 1e-8
    assert abs(st["residual"] - ref["residual"]) <= 1e-8


def test_csc_invalid_arguments(P, w8):
    s, S, oa, H0, gamma, q_ref, z, w = w8
    h = P.tb_create_system(s)
    for kw in ({"mix": 0.0}, {"mix": 1.5}, {"scf_tol": 0.0}, {"max_scf": 0}):
        with pytest.raises(P.TBError):
            P.tb_csc_loop(h, z[:4], w[:4], gamma, q_ref, copts=P.tb_default_csc_opts(**kw))
    with pytest.raises(ValueError):
        P.tb_csc_hamiltonian(h, gamma[:3], np.zeros(s.n_atoms))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_csc_forces_match_oracle(P, w8, w8_loop, prec):
    """Forces of the charge-self-consistent model on the device
    (tb_csc_forces) against the oracle's scc_forces at the oracle loop's
    self-consistent dq: every component to 1e-7 of the largest, zero net
    force; the handle is left at H0 + H^CSC(dq)."""
    from tbinputs import overlap_bond_derivatives, klopman_ohno_gamma_gradient
    s, S, oa, H0, gamma, q_ref, z, w = w8
    dq = w8_loop["dq"]
    dS = overlap_bond_derivatives(s)
    dg = 0.25 * klopman_ohno_gamma_gradient(s)
    ref = csc.scc_forces(H0, S, oa, gamma, dg, q_ref, dq, z, w, dS, s.orb_per_atom, s.brow_ptr, s.bcol, s.eps, s.K)
    h = P.tb_create_system(s)
    F, st = P.tb_csc_forces(h, z, w, gamma, dg, dq, dS, opts=P.tb_default_opts(precision=prec))
    assert st["status"] == "TB_OK"
    scale = np.abs(ref).max()
    assert np.abs(F - ref).max() <= 1e-7 * scale
    assert np.abs(F.sum(axis=0)).max() <= 1e-8 * scale
    q, _ = P.tb_mulliken_charges(h, z, w, opts=P.tb_default_opts(precision=prec))
    assert np.abs(q.cpu().numpy() - w8_loop["q"]).max() <= 1e-7


def test_csc_forces_without_coulomb_gradient_differ(P, w8, w8_loop):
    """The Coulomb-gradient term matters: with dgamma = 0 the device forces
    equal the oracle's forces without that term and differ from the full
    ones."""
    from tbinputs import overlap_bond_derivatives, klopman_ohno_gamma_gradient
    s, S, oa, H0, gamma, q_ref, z, w = w8
    dq = w8_loop["dq"]
    dS = overlap_bond_derivatives(s)
    dg = 0.25 * klopman_ohno_gamma_gradient(s)
    h = P.tb_create_system(s)
    F0, _ = P.tb_csc_forces(h, z, w, gamma, np.zeros_like(dg), dq, dS)
    ref0 = csc.scc_forces(H0, S, oa, gamma, np.zeros_like(dg), q_ref, dq, z, w, dS, s.orb_per_atom, s.brow_ptr,
                          s.bcol, s.eps, s.K)
    full = csc.scc_forces(H0, S, oa, gamma, dg, q_ref, dq, z, w, dS, s.orb_per_atom, s.brow_ptr, s.bcol, s.eps, s.K)
    assert np.abs(F0 - ref0).max() <= 1e-7 * np.abs(ref0).max()
    assert np.abs(F0 - full).max() > 1e-4 * np.abs(full).max()

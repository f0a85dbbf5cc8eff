"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; host-side validation returns the documented status codes
(no GPU needed: tb_create validates before touching the device)."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from tbinputs import si_system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1002_1202_gb300 import _build_lib, tb
    _build_lib.build()
    return tb.load_library()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(tb_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    from paper_1002_1202_gb300 import tb
    declared = _declared()
    assert len(declared) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", tb.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tb_\w+)", out))
    assert declared <= exported, declared - exported
    for name in declared:
        assert hasattr(lib, name)
    assert declared == {s[0] for s in tb.SIGNATURES}


def test_status_strings(lib):
    from paper_1002_1202_gb300 import tb
    assert tb.tb_status_string(0) == "TB_OK"
    assert tb.tb_status_string(6) == "TB_ERR_NOT_CONVERGED"
    assert tb.tb_status_string(123) == "TB_UNKNOWN_STATUS"


def test_default_opts(lib):
    from paper_1002_1202_gb300 import tb
    o = tb.tb_default_opts()
    assert o.tol == 1e-10 and o.inner_tol == 1e-13 and o.switching == 1 and o.seed == 0


@pytest.fixture(scope="module")
def si():
    return si_system()


def _create(s, **over):
    from paper_1002_1202_gb300 import tb
    args = dict(orb_per_atom=s.orb_per_atom, brow_ptr=s.brow_ptr, bcol=s.bcol, S_vals=s.S_vals, H_vals=None,
                eps=s.eps, K=s.K)
    args.update(over)
    return tb.tb_create(**args, stream=0)


def _status(fn):
    from paper_1002_1202_gb300 import tb
    try:
        fn()
    except tb.TBError as e:
        return e.status
    return 0


@pytest.mark.parametrize("case,want", [
    ("bad_col", 1), ("unsorted", 1), ("no_diag", 1), ("bad_orb", 1), ("ptr", 1),
    ("asym_value", 2), ("asym_pattern", 2), ("neg_diag", 3), ("nan", 1),
])
def test_create_validation(lib, si, case, want):
    s = si
    if case == "bad_col":
        bc = s.bcol.copy(); bc[5] = s.n_atoms + 3
        st = _status(lambda: _create(s, bcol=bc))
    elif case == "unsorted":
        bc = s.bcol.copy(); b0 = s.brow_ptr[2]; bc[b0], bc[b0 + 1] = bc[b0 + 1], bc[b0]
        st = _status(lambda: _create(s, bcol=bc))
    elif case == "no_diag":
        # drop atom 0's diagonal block from its row (and keep the pattern consistent in length)
        bc = s.bcol.copy(); row = bc[s.brow_ptr[0]:s.brow_ptr[1]]
        assert row[0] == 0
        bc[s.brow_ptr[0]] = -1
        st = _status(lambda: _create(s, bcol=bc))
    elif case == "bad_orb":
        o = s.orb_per_atom.copy(); o[3] = 2
        st = _status(lambda: _create(s, orb_per_atom=o))
    elif case == "ptr":
        bp = s.brow_ptr.copy(); bp[4], bp[5] = bp[5], bp[4]
        st = _status(lambda: _create(s, brow_ptr=bp))
    elif case == "asym_value":
        sv = s.S_vals.copy(); sv[16 * 1 + 2] += 1e-4
        st = _status(lambda: _create(s, S_vals=sv))
    elif case == "asym_pattern":
        # remove block (0, j) but keep (j, 0): pattern no longer symmetric
        keep = np.ones(s.nb, dtype=bool)
        b = s.brow_ptr[0] + 1
        keep[b] = False
        bp = s.brow_ptr.copy(); bp[1:] -= 1
        sv = np.delete(s.S_vals, np.arange(16 * b, 16 * b + 16))
        st = _status(lambda: _create(s, brow_ptr=bp, bcol=s.bcol[keep], S_vals=sv))
    elif case == "neg_diag":
        sv = s.S_vals.copy()
        b = int(s.brow_ptr[0])   # block (0, 0)
        sv[16 * b] = -1.0
        st = _status(lambda: _create(s, S_vals=sv))
    elif case == "nan":
        e = s.eps.copy(); e[7] = np.nan
        st = _status(lambda: _create(s, eps=e))
    assert st == want


def test_create_without_device_reports_no_device(lib, si):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _status(lambda: _create(si)) == 9


def test_csc_defaults_and_null_arguments(lib):
    import ctypes as C
    from paper_1002_1202_gb300 import tb
    o = tb.CscOpts()
    lib.tb_default_csc_opts(C.byref(o))
    assert (o.max_scf, o.scf_tol, o.mix) == (50, 1e-6, 0.3)
    so = tb.SolveOpts()
    lib.tb_default_opts(C.byref(so))
    st = tb.CscStats()
    z = np.array([0.0, 1.0])
    zp = z.ctypes.data_as(C.POINTER(C.c_double))
    # a NULL handle is rejected before any device work
    assert lib.tb_csc_hamiltonian(None, None, None, None) == 1
    assert lib.tb_csc_loop(None, 1, zp, zp, 2.0, None, None, None, C.byref(o), C.byref(so), None, None,
                           C.byref(st), None) == 1


def test_batch_validation(lib, si):
    """tb_create_batch checks every system as tb_create does and rejects
    batches that mix explicit and ASED Hamiltonians or ASED constants."""
    import dataclasses
    import torch
    from paper_1002_1202_gb300 import tb
    other_K = dataclasses.replace(si, K=si.K + 0.5)
    assert _status(lambda: tb.tb_create_batch([si, other_K], stream=0)) == 1
    bad = dataclasses.replace(si, bcol=si.bcol.copy())
    bad.bcol[3] = si.n_atoms + 1
    assert _status(lambda: tb.tb_create_batch([si, bad], stream=0)) == 1
    assert _status(lambda: tb.tb_create_batch([], stream=0)) == 1
    if not torch.cuda.is_available():
        assert _status(lambda: tb.tb_create_batch([si, si], stream=0)) == 9


def test_mulliken_vjp_null_arguments(lib):
    import ctypes as C
    from paper_1002_1202_gb300 import tb
    so = tb.SolveOpts()
    lib.tb_default_opts(C.byref(so))
    z = np.array([0.0, 1.0])
    zp = z.ctypes.data_as(C.POINTER(C.c_double))
    assert lib.tb_mulliken_vjp(None, 1, zp, zp, 2.0, None, C.byref(so), None, None, None, None) == 1

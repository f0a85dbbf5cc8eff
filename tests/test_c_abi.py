"""The C ABI from C: tests/c_abi/dimer.c compiled as C99 against
include/tbcocg.h and linked to libtbcocg.so.  Without a GPU it checks the
host-only calls and that tb_create reports TB_ERR_NO_DEVICE; on a GPU it
also solves the two-atom dimer and compares the Mulliken populations with
their closed form (the closed form itself is pinned here against the
oracle)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    from paper_1002_1202_gb300 import _build_lib
    _build_lib.build()
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    libdir = os.path.dirname(_build_lib.LIB)
    out = str(tmp_path_factory.mktemp("cabi") / "dimer")
    r = subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi", "dimer.c"), "-o", out, "-L", libdir, "-ltbcocg",
                        "-Wl,-rpath," + libdir, "-lm"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def test_dimer_closed_form_against_oracle():
    """The program's closed form for the dimer populations equals the
    oracle's dense Mulliken populations on the same inputs."""
    from oracle import dense
    s, eps, K, g_s = 0.35, -13.6, 1.75, 2.0
    S = np.array([[1.0, s], [s, 1.0]])
    H = dense.ased_hamiltonian(S, np.array([eps, eps]), K, np.array([0, 1]))
    NK = 32
    dx = 35.0 / (NK - 1)
    z = np.array([-30.0 + k * dx + 0.5j for k in range(NK)])
    w = np.array([0.5 * dx if k in (0, NK - 1) else dx for k in range(NK)])
    q = dense.mulliken_orbital(H, S, z, w, g_s)
    hb = K * eps * s
    ev = [(eps + hb) / (1 + s), (eps - hb) / (1 - s)]
    ref = 0.5 * g_s * sum(-np.imag(np.sum(w / (z - e))) / math.pi for e in ev)
    assert np.abs(q - ref).max() <= 1e-12 * abs(ref)


def test_c_program_runs(exe):
    import torch
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    want = "ok" if torch.cuda.is_available() else "no-device"
    assert r.returncode == 0 and r.stdout.strip() == want, (r.returncode, r.stdout, r.stderr)


def test_struct_layouts_match_the_binding(tmp_path):
    """sizeof and offsetof of every C-ABI struct, printed by a C program
    compiled against the header, equal those of the ctypes mirrors."""
    import ctypes
    from paper_1002_1202_gb300 import tb
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    out = str(tmp_path / "layout")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi", "layout.c"), "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lines = subprocess.run([out], capture_output=True, text=True, check=True).stdout.split("\n")
    mirrors = {"tb_system_desc": tb.SystemDesc, "tb_solve_opts": tb.SolveOpts, "tb_stats": tb.Stats,
               "tb_csc_opts": tb.CscOpts, "tb_csc_stats": tb.CscStats, "tb_tune": tb.Tune}
    seen = set()
    for ln in filter(None, lines):
        name, field, value = ln.split()
        cls = mirrors[name]
        if field == "sizeof":
            assert ctypes.sizeof(cls) == int(value), name
        else:
            assert getattr(cls, field).offset == int(value), (name, field)
            seen.add((name, field))
    for name, cls in mirrors.items():
        assert {f for f, _ in cls._fields_} == {f for n, f in seen if n == name}, name



@pytest.mark.gpu
def test_c_program_solves_dimer_on_gpu(exe):
    """The same C99 program on a GPU: the two-atom solve through the plain C
    ABI must print ok (its populations equal their closed form)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)

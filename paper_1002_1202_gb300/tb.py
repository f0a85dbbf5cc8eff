"""Python binding of the C ABI in ``include/tbcocg.h`` (ctypes, marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it converts numpy/torch arguments to pointers and
sizes, calls the library, and turns the status into an exception.  Device
outputs are torch tensors (PyTorch is used for device memory and streams);
host outputs are numpy arrays.  The library must be built
(``paper_1002_1202_gb300._build_lib.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build_lib

TB_OK = 0
TB_ERR_NOT_CONVERGED = 6
TB_FP64 = 0
TB_MIXED = 1

_STATUS = {
    0: "TB_OK", 1: "TB_ERR_INVALID_ARG", 2: "TB_ERR_NOT_SYMMETRIC", 3: "TB_ERR_S_NOT_SPD",
    4: "TB_ERR_OOM", 5: "TB_ERR_CUDA", 6: "TB_ERR_NOT_CONVERGED", 7: "TB_ERR_BREAKDOWN",
    8: "TB_ERR_TIMEOUT", 9: "TB_ERR_NO_DEVICE", 10: "TB_ERR_TOO_LARGE",
}


class TBError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)}")


class SystemDesc(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int32),
        ("orb_per_atom", C.POINTER(C.c_int32)),
        ("brow_ptr", C.POINTER(C.c_int64)),
        ("bcol", C.POINTER(C.c_int32)),
        ("S_vals", C.POINTER(C.c_double)),
        ("H_vals", C.POINTER(C.c_double)),
        ("eps", C.POINTER(C.c_double)),
        ("K", C.c_double),
        ("precision", C.c_int32),
    ]


TB_INNER_CHEBYSHEV = 0
TB_INNER_CG = 1


class SolveOpts(C.Structure):
    _fields_ = [
        ("tol", C.c_double),
        ("inner_tol", C.c_double),
        ("max_iter", C.c_int32),
        ("inner_max_iter", C.c_int32),
        ("panel", C.c_int32),
        ("seed", C.c_int32),
        ("switching", C.c_int32),
        ("force_switch_every", C.c_int32),
        ("precision", C.c_int32),
        ("inner_lo_tol", C.c_double),
        ("inner_method", C.c_int32),
        ("state_bytes", C.c_int64),
    ]


class Tune(C.Structure):
    _fields_ = [
        ("panel", C.c_int32),
        ("streams", C.c_int32),
        ("cheb_cpt", C.c_int32),
        ("ctas_per_sm", C.c_int32),
        ("rate", C.c_double),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("conv_iter", C.POINTER(C.c_int32)),
        ("outer_iterations", C.c_int64),
        ("inner_iterations", C.c_int64),
        ("max_column_iterations", C.c_int64),
        ("switches", C.c_int32),
        ("unconverged", C.c_int32),
        ("seconds", C.c_double),
        ("inner_redos", C.c_int32),
    ]


class CscOpts(C.Structure):
    _fields_ = [
        ("max_scf", C.c_int32),
        ("scf_tol", C.c_double),
        ("mix", C.c_double),
    ]


class CscStats(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32),
        ("residual", C.c_double),
        ("outer_iterations", C.c_int64),
        ("inner_iterations", C.c_int64),
        ("seconds", C.c_double),
    ]


# (name, restype, argtypes) of every entry point declared in include/tbcocg.h
_VP = C.c_void_p
_DP = C.POINTER(C.c_double)
_I32P = C.POINTER(C.c_int32)
_I64P = C.POINTER(C.c_int64)
SIGNATURES = [
    ("tb_create", C.c_int, [C.POINTER(_VP), C.POINTER(SystemDesc), _VP]),
    ("tb_destroy", C.c_int, [_VP]),
    ("tb_create_batch", C.c_int, [C.POINTER(_VP), C.POINTER(SystemDesc), C.c_int32, _VP]),
    ("tb_num_systems", C.c_int32, [_VP]),
    ("tb_batch_offsets", C.c_int, [_VP, _I64P, _I64P]),
    ("tb_num_orbitals", C.c_int64, [_VP]),
    ("tb_num_atoms", C.c_int64, [_VP]),
    ("tb_num_blocks", C.c_int64, [_VP]),
    ("tb_default_opts", None, [C.POINTER(SolveOpts)]),
    ("tb_shifted_cocg", C.c_int, [_VP, C.c_int32, _DP, C.c_int32, _I32P, C.POINTER(SolveOpts), _VP,
                                  C.POINTER(Stats), _VP]),
    ("tb_green_elements", C.c_int, [_VP, C.c_int32, _DP, C.c_int32, _I32P, _I64P, _I32P,
                                    C.POINTER(SolveOpts), _VP, C.POINTER(Stats), _VP]),
    ("tb_green_elements_dz", C.c_int, [_VP, C.c_int32, _DP, C.c_int32, _I32P, _I64P, _I32P,
                                       C.POINTER(SolveOpts), _VP, _VP, C.POINTER(Stats), _VP]),
    ("tb_band_energy", C.c_int, [_VP, C.c_int32, _DP, _DP, C.c_double, C.POINTER(SolveOpts), _VP, _VP, _VP,
                                 C.POINTER(Stats), _VP]),
    ("tb_forces", C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("tb_overlap_bounds", C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("tb_overlap_bounds_desc", C.c_int, [C.POINTER(SystemDesc), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("tb_chebyshev_plan", C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_double), C.POINTER(C.c_float), C.c_int32]),
    ("tb_mulliken_vjp", C.c_int, [_VP, C.c_int32, _DP, _DP, C.c_double, _VP, C.POINTER(SolveOpts), _VP, _VP,
                                  C.POINTER(Stats), _VP]),
    ("tb_mulliken_orbital", C.c_int, [_VP, C.c_int32, _DP, _DP, C.c_double, C.c_int32, _I32P,
                                      C.POINTER(SolveOpts), _VP, C.POINTER(Stats), _VP]),
    ("tb_mulliken_charges", C.c_int, [_VP, C.c_int32, _DP, _DP, C.c_double, C.POINTER(SolveOpts), _VP,
                                      C.POINTER(Stats), _VP]),
    ("tb_default_csc_opts", None, [C.POINTER(CscOpts)]),
    ("tb_csc_hamiltonian", C.c_int, [_VP, _VP, _VP, _VP]),
    ("tb_csc_loop", C.c_int, [_VP, C.c_int32, _DP, _DP, C.c_double, _VP, _VP, _VP, C.POINTER(CscOpts),
                              C.POINTER(SolveOpts), _VP, _VP, C.POINTER(CscStats), _VP]),
    ("tb_generalized_lanczos", C.c_int, [_VP, C.c_int32, C.c_int32, C.c_double, _VP, _VP, _VP, _VP]),
    ("tb_lanczos_green", C.c_int, [_VP, _VP, C.c_double, C.c_int32, C.c_int32, _DP, _VP, _VP]),
    ("tb_lanczos_green_batch", C.c_int, [C.c_int32, _VP, _VP, _VP, C.c_int32, C.c_int32, _DP, _VP, _VP]),
    ("tb_generalized_lanczos_batch", C.c_int, [_VP, C.c_int32, _I32P, C.c_int32, C.POINTER(SolveOpts), _VP, _VP,
                                               _VP, _VP]),
    ("tb_generalized_lanczos_noalloc", C.c_int, [_VP, C.c_int32, C.c_int32, C.c_double, _VP, _VP, _VP, _VP]),
    ("tb_autotune", C.c_int, [_VP, C.c_int32, _DP, _DP, C.c_double, C.POINTER(SolveOpts), C.c_int32,
                              C.POINTER(Tune), C.c_int32, C.POINTER(C.c_int32), _VP]),
    ("tb_csc_forces", C.c_int, [_VP, C.c_int32, _DP, _DP, C.c_double, _VP, _VP, _VP, _VP, C.POINTER(SolveOpts),
                                _VP, C.POINTER(Stats), _VP]),
    ("tb_measure_fma_peak", C.c_int, [C.c_int32, _DP, _VP]),
    ("tb_status_string", C.c_char_p, [C.c_int]),
    ("tb_launch_count", C.c_int64, []),
    ("tb_profile_enable", None, [C.c_int32]),
    ("tb_profile_read", C.c_int, [C.c_int32, _I64P, _DP]),
    ("tb_profile_busy", C.c_int, [C.c_int32, _DP]),
]

KERNELS = {"inner_spmv": 0, "inner_update": 1, "outer_spmm": 2, "outer_update": 3, "finish": 4,
           "shift_step": 5, "full_update": 6, "other": 7, "inner32_spmv": 8, "inner32_update": 9,
           "refine_residual": 10, "refine_aux": 11, "csc": 12, "inner32_cheb": 13}

_lib = None


def library_path() -> str:
    return _build_lib.LIB


def load_library(path: str | None = None) -> C.CDLL:
    """Load libtbcocg.so (building nothing); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build_lib.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_1002_1202_gb300._build_lib.build()")
    lib = C.CDLL(p)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _stream(stream):
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return C.c_void_p(0)
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _complex_host(z) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(z, dtype=np.complex128)).view(np.float64)


def _out_ptr(out):
    if isinstance(out, np.ndarray):
        if not out.flags.c_contiguous:
            raise ValueError("output array must be contiguous")
        return C.c_void_p(out.ctypes.data)
    if not out.is_contiguous():
        raise ValueError("output tensor must be contiguous")
    return C.c_void_p(out.data_ptr())


def _check(st: int, where: str, allow_unconverged: bool):
    if st == TB_OK or (st == TB_ERR_NOT_CONVERGED and allow_unconverged):
        return st
    raise TBError(st, where)


def tb_default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    load_library().tb_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Handle:
    """A device copy of a block-sparse system (tb_create / tb_destroy)."""

    def __init__(self, ptr: C.c_void_p, n_orb: int, n_atoms: int, nb: int):
        self.ptr = ptr
        self.n_orb = n_orb
        self.n_atoms = n_atoms
        self.nb = nb

    def close(self):
        if self.ptr:
            load_library().tb_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tb_create(orb_per_atom, brow_ptr, bcol, S_vals, H_vals=None, eps=None, K=1.75, stream=None) -> Handle:
    lib = load_library()
    orb = np.ascontiguousarray(orb_per_atom, dtype=np.int32)
    bp = np.ascontiguousarray(brow_ptr, dtype=np.int64)
    bc = np.ascontiguousarray(bcol, dtype=np.int32)
    sv = np.ascontiguousarray(S_vals, dtype=np.float64)
    hv = None if H_vals is None else np.ascontiguousarray(H_vals, dtype=np.float64)
    ev = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    d = SystemDesc()
    d.n_atoms = len(orb)
    d.orb_per_atom = _ptr(orb, C.c_int32)
    d.brow_ptr = _ptr(bp, C.c_int64)
    d.bcol = _ptr(bc, C.c_int32)
    d.S_vals = _ptr(sv, C.c_double)
    d.H_vals = _ptr(hv, C.c_double) if hv is not None else None
    d.eps = _ptr(ev, C.c_double) if ev is not None else None
    d.K = float(K)
    d.precision = TB_FP64
    h = C.c_void_p()
    _check(lib.tb_create(C.byref(h), C.byref(d), _stream(stream)), "tb_create", False)
    return Handle(h, int(lib.tb_num_orbitals(h)), int(lib.tb_num_atoms(h)), int(lib.tb_num_blocks(h)))


def tb_create_batch(systems, stream=None) -> Handle:
    """tb_create_batch from a list of ``tbinputs.TBSystem`` (H by Eq. Hap-1;
    all K equal).  The handle gets ``atom_off`` and ``orb_off`` (numpy int64
    [n_systems + 1]): the first atom and orbital of every system."""
    lib = load_library()
    keep = []
    descs = (SystemDesc * len(systems))()
    for d, so in zip(descs, systems):
        arrs = [np.ascontiguousarray(so.orb_per_atom, dtype=np.int32),
                np.ascontiguousarray(so.brow_ptr, dtype=np.int64),
                np.ascontiguousarray(so.bcol, dtype=np.int32),
                np.ascontiguousarray(so.S_vals, dtype=np.float64),
                np.ascontiguousarray(so.eps, dtype=np.float64)]
        keep.append(arrs)
        d.n_atoms = len(arrs[0])
        d.orb_per_atom = _ptr(arrs[0], C.c_int32)
        d.brow_ptr = _ptr(arrs[1], C.c_int64)
        d.bcol = _ptr(arrs[2], C.c_int32)
        d.S_vals = _ptr(arrs[3], C.c_double)
        d.H_vals = None
        d.eps = _ptr(arrs[4], C.c_double)
        d.K = float(so.K)
        d.precision = TB_FP64
    h = C.c_void_p()
    _check(lib.tb_create_batch(C.byref(h), descs, len(systems), _stream(stream)), "tb_create_batch", False)
    out = Handle(h, int(lib.tb_num_orbitals(h)), int(lib.tb_num_atoms(h)), int(lib.tb_num_blocks(h)))
    ns = int(lib.tb_num_systems(h))
    out.atom_off = np.zeros(ns + 1, dtype=np.int64)
    out.orb_off = np.zeros(ns + 1, dtype=np.int64)
    _check(lib.tb_batch_offsets(h, _ptr(out.atom_off, C.c_int64), _ptr(out.orb_off, C.c_int64)),
           "tb_batch_offsets", False)
    return out


def tb_create_system(sysobj, explicit_H=None, stream=None) -> Handle:
    """tb_create from a ``tbinputs.TBSystem`` (H by Eq. Hap-1 unless given)."""
    return tb_create(sysobj.orb_per_atom, sysobj.brow_ptr, sysobj.bcol, sysobj.S_vals, explicit_H, sysobj.eps,
                     sysobj.K, stream)


def _stats(R: int, K: int, want_conv: bool):
    st = Stats()
    conv = None
    if want_conv:
        conv = np.full(R * K, -1, dtype=np.int32)
        st.conv_iter = _ptr(conv, C.c_int32)
    return st, conv


def _stats_dict(st: Stats, conv, R, K, status):
    return {"status": _STATUS.get(status, status), "outer_iterations": st.outer_iterations,
            "inner_iterations": st.inner_iterations, "max_column_iterations": st.max_column_iterations,
            "switches": st.switches, "unconverged": st.unconverged, "seconds": st.seconds,
            "inner_redos": st.inner_redos,
            "conv_iter": None if conv is None else conv.reshape(R, K)}


def tb_shifted_cocg(h: Handle, z, cols, opts: SolveOpts | None = None, out=None, stream=None,
                    allow_unconverged=False):
    """Full solutions x[k, c, :] = (z_k S - H)^-1 e_{cols[c]}; returns (out, stats)."""
    import torch
    zz = _complex_host(z)
    cc = np.ascontiguousarray(cols, dtype=np.int32)
    K, R = len(zz) // 2, len(cc)
    if out is None:
        out = torch.empty((K, R, h.n_orb), dtype=torch.complex128, device="cuda")
    opts = opts or tb_default_opts()
    st, conv = _stats(R, K, True)
    s = load_library().tb_shifted_cocg(h.ptr, K, _ptr(zz, C.c_double), R, _ptr(cc, C.c_int32), C.byref(opts),
                                       _out_ptr(out), C.byref(st), _stream(stream))
    _check(s, "tb_shifted_cocg", allow_unconverged)
    return out, _stats_dict(st, conv, R, K, s)


def tb_green_elements(h: Handle, z, cols, row_ptr, rows, opts: SolveOpts | None = None, out=None, stream=None,
                      allow_unconverged=False):
    """G[(row_ptr[c]+r), k] = G_{rows[row_ptr[c]+r], cols[c]}(z_k); returns (out, stats)."""
    import torch
    zz = _complex_host(z)
    cc = np.ascontiguousarray(cols, dtype=np.int32)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    rr = np.ascontiguousarray(rows, dtype=np.int32)
    K, R = len(zz) // 2, len(cc)
    if out is None:
        out = torch.empty((int(rp[-1]), K), dtype=torch.complex128, device="cuda")
    opts = opts or tb_default_opts()
    st, conv = _stats(R, K, True)
    s = load_library().tb_green_elements(h.ptr, K, _ptr(zz, C.c_double), R, _ptr(cc, C.c_int32),
                                         _ptr(rp, C.c_int64), _ptr(rr, C.c_int32), C.byref(opts), _out_ptr(out),
                                         C.byref(st), _stream(stream))
    _check(s, "tb_green_elements", allow_unconverged)
    return out, _stats_dict(st, conv, R, K, s)


def tb_green_elements_dz(h: Handle, z, cols, row_ptr, rows, opts: SolveOpts | None = None, out=None, dout=None,
                         stream=None, allow_unconverged=False):
    """As tb_green_elements, plus dG/dz at the same elements; returns
    (G, dG, stats)."""
    import torch
    zz = _complex_host(z)
    cc = np.ascontiguousarray(cols, dtype=np.int32)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    rr = np.ascontiguousarray(rows, dtype=np.int32)
    K, R = len(zz) // 2, len(cc)
    if out is None:
        out = torch.empty((int(rp[-1]), K), dtype=torch.complex128, device="cuda")
    if dout is None:
        dout = torch.empty((int(rp[-1]), K), dtype=torch.complex128, device="cuda")
    opts = opts or tb_default_opts()
    st, conv = _stats(R, K, True)
    s = load_library().tb_green_elements_dz(h.ptr, K, _ptr(zz, C.c_double), R, _ptr(cc, C.c_int32),
                                            _ptr(rp, C.c_int64), _ptr(rr, C.c_int32), C.byref(opts), _out_ptr(out),
                                            _out_ptr(dout), C.byref(st), _stream(stream))
    _check(s, "tb_green_elements_dz", allow_unconverged)
    return out, dout, _stats_dict(st, conv, R, K, s)


def tb_band_energy(h: Handle, z, w, g_s=2.0, opts: SolveOpts | None = None, n_values=None, stream=None,
                   allow_unconverged=False):
    """Band energy E and dE/dH, dE/dS in the caller's block layout (length
    ``n_values`` = len(S_vals)); returns (E, dE_dH, dE_dS, stats) as numpy."""
    zz = _complex_host(z)
    ww = _complex_host(w)
    K = len(zz) // 2
    if n_values is None:
        raise ValueError("n_values (the length of the S_vals array) is required")
    E = np.zeros(1)
    gH = np.zeros(int(n_values))
    gS = np.zeros(int(n_values))
    opts = opts or tb_default_opts()
    st, _ = _stats(h.n_orb, K, False)
    s = load_library().tb_band_energy(h.ptr, K, _ptr(zz, C.c_double), _ptr(ww, C.c_double), float(g_s),
                                      C.byref(opts), _out_ptr(E), _out_ptr(gH), _out_ptr(gS), C.byref(st),
                                      _stream(stream))
    _check(s, "tb_band_energy", allow_unconverged)
    return float(E[0]), gH, gS, _stats_dict(st, None, h.n_orb, K, s)


def tb_overlap_bounds(h: Handle):
    """(lo, hi): the bounds of the spectrum of S used by the Chebyshev
    corrections of the mixed-precision inner solve."""
    lo, hi = C.c_double(), C.c_double()
    _check(load_library().tb_overlap_bounds(h.ptr, C.byref(lo), C.byref(hi)), "tb_overlap_bounds", False)
    return lo.value, hi.value


def tb_overlap_bounds_desc(system):
    """(lo, hi) of ``tb_overlap_bounds`` for a ``tbinputs.TBSystem`` (or any
    object with orb_per_atom, brow_ptr, bcol, S_vals), on the host only."""
    arrs = [np.ascontiguousarray(system.orb_per_atom, dtype=np.int32),
            np.ascontiguousarray(system.brow_ptr, dtype=np.int64),
            np.ascontiguousarray(system.bcol, dtype=np.int32),
            np.ascontiguousarray(system.S_vals, dtype=np.float64)]
    d = SystemDesc()
    d.n_atoms = len(arrs[0])
    d.orb_per_atom = _ptr(arrs[0], C.c_int32)
    d.brow_ptr = _ptr(arrs[1], C.c_int64)
    d.bcol = _ptr(arrs[2], C.c_int32)
    d.S_vals = _ptr(arrs[3], C.c_double)
    d.H_vals = None
    d.eps = None
    d.K = 0.0
    d.precision = TB_FP64
    lo, hi = C.c_double(), C.c_double()
    _check(load_library().tb_overlap_bounds_desc(C.byref(d), C.byref(lo), C.byref(hi)), "tb_overlap_bounds_desc",
           False)
    return lo.value, hi.value


def tb_chebyshev_plan(lo, hi, lo_tol=1e-6, inner_tol=1e-13, cap=1000):
    """dict(n, n_last, rounds, gamma, omega) of the mixed path's Chebyshev
    corrections for spectrum bounds [lo, hi] (host only)."""
    n, nl, r = C.c_int32(), C.c_int32(), C.c_int32()
    g = C.c_double()
    om = np.zeros(max(1, int(cap)), dtype=np.float32)
    _check(load_library().tb_chebyshev_plan(float(lo), float(hi), float(lo_tol), float(inner_tol), int(cap),
                                            C.byref(n), C.byref(nl), C.byref(r), C.byref(g),
                                            om.ctypes.data_as(C.POINTER(C.c_float)), len(om)),
           "tb_chebyshev_plan", False)
    return {"n": n.value, "n_last": nl.value, "rounds": r.value, "gamma": g.value, "omega": om[:n.value].copy()}


def tb_mulliken_vjp(h: Handle, z, w, v, n_values: int, g_s=2.0, opts: SolveOpts | None = None, stream=None,
                    allow_unconverged=False):
    """dL/dH, dL/dS (caller block layout, length n_values) of
    L = sum_a v_a q_a; returns (dL_dH, dL_dS, stats) as numpy."""
    keep = []
    zz = _complex_host(z)
    ww = _complex_host(w)
    K = len(zz) // 2
    gH = np.zeros(int(n_values))
    gS = np.zeros(int(n_values))
    opts = opts or tb_default_opts()
    st, _ = _stats(h.n_orb, K, False)
    s = load_library().tb_mulliken_vjp(h.ptr, K, _ptr(zz, C.c_double), _ptr(ww, C.c_double), float(g_s),
                                       _in_ptr(v, h.n_orb, keep), C.byref(opts), _out_ptr(gH), _out_ptr(gS),
                                       C.byref(st), _stream(stream))
    _check(s, "tb_mulliken_vjp", allow_unconverged)
    return gH, gS, _stats_dict(st, None, h.n_orb, K, s)


def tb_forces(h: Handle, dE_dH, dE_dS, dS_dd, dH_dd=None, stream=None):
    """Forces (n_atoms, 3) from band-energy gradients and geometry
    derivatives (3, n_values); dH_dd None: the Eq. Hap-1 rule."""
    keep = []
    nv = len(dE_dH)
    F = np.zeros((h.n_atoms, 3))
    s = load_library().tb_forces(h.ptr, _in_ptr(dE_dH, nv, keep), _in_ptr(dE_dS, nv, keep),
                                 _in_ptr(np.ravel(dS_dd), 3 * nv, keep),
                                 _in_ptr(None if dH_dd is None else np.ravel(dH_dd), 3 * nv, keep),
                                 _out_ptr(F), _stream(stream))
    _check(s, "tb_forces", False)
    return F


def tb_mulliken_orbital(h: Handle, z, w, cols, g_s=2.0, opts: SolveOpts | None = None, out=None, stream=None,
                        allow_unconverged=False):
    """Gross Mulliken populations of the orbitals ``cols``; returns (out, stats)."""
    import torch
    zz = _complex_host(z)
    ww = _complex_host(w)
    cc = np.ascontiguousarray(cols, dtype=np.int32)
    K, R = len(zz) // 2, len(cc)
    if out is None:
        out = torch.empty((R,), dtype=torch.float64, device="cuda")
    opts = opts or tb_default_opts()
    st, conv = _stats(R, K, True)
    s = load_library().tb_mulliken_orbital(h.ptr, K, _ptr(zz, C.c_double), _ptr(ww, C.c_double), float(g_s), R,
                                           _ptr(cc, C.c_int32), C.byref(opts), _out_ptr(out), C.byref(st),
                                           _stream(stream))
    _check(s, "tb_mulliken_orbital", allow_unconverged)
    return out, _stats_dict(st, conv, R, K, s)


def tb_mulliken_charges(h: Handle, z, w, g_s=2.0, opts: SolveOpts | None = None, out=None, stream=None,
                        allow_unconverged=False):
    """Gross Mulliken population of every atom; returns (out, stats)."""
    import torch
    zz = _complex_host(z)
    ww = _complex_host(w)
    K = len(zz) // 2
    if out is None:
        out = torch.empty((h.n_atoms,), dtype=torch.float64, device="cuda")
    opts = opts or tb_default_opts()
    st, _ = _stats(h.n_orb, K, False)
    s = load_library().tb_mulliken_charges(h.ptr, K, _ptr(zz, C.c_double), _ptr(ww, C.c_double), float(g_s),
                                           C.byref(opts), _out_ptr(out), C.byref(st), _stream(stream))
    _check(s, "tb_mulliken_charges", allow_unconverged)
    return out, _stats_dict(st, None, h.n_orb, K, s)


def tb_csc_forces(h: Handle, z, w, gamma, dgamma, dq, dS_dd, g_s=2.0, opts: SolveOpts | None = None, out=None,
                  stream=None, allow_unconverged=False):
    """Forces (n_atoms, 3) of the charge-self-consistent model at the
    self-consistent dq (tb_csc_loop's dq_out): gamma (n, n), dgamma (n, n, 3)
    = d gamma_Ik / d R_I, dS_dd (3, n_values); returns (F, stats)."""
    keep = []
    zz = _complex_host(z)
    ww = _complex_host(w)
    K = len(zz) // 2
    n = h.n_atoms
    if out is None:
        out = np.zeros((n, 3))
    opts = opts or tb_default_opts()
    st, _ = _stats(h.n_orb, K, False)
    s = load_library().tb_csc_forces(h.ptr, K, _ptr(zz, C.c_double), _ptr(ww, C.c_double), float(g_s),
                                     _in_ptr(gamma, n * n, keep), _in_ptr(dgamma, n * n * 3, keep),
                                     _in_ptr(dq, n, keep), _in_ptr(dS_dd, _numel(dS_dd), keep), C.byref(opts),
                                     _out_ptr(out), C.byref(st), _stream(stream))
    _check(s, "tb_csc_forces", allow_unconverged)
    return out, _stats_dict(st, None, h.n_orb, K, s)


def tb_autotune(h: Handle, z, w, g_s=2.0, opts: SolveOpts | None = None, iters=3, stream=None) -> list:
    """Time the launch choices (panel width, panels in flight, Chebyshev-step
    form) for this handle and shift set; the best is kept in the handle for
    later calls with panel 0.  Returns the candidates as dicts, best first."""
    zz = _complex_host(z)
    ww = _complex_host(w)
    K = len(zz) // 2
    opts = opts or tb_default_opts()
    out = (Tune * 32)()
    n = C.c_int32(0)
    s = load_library().tb_autotune(h.ptr, K, _ptr(zz, C.c_double), _ptr(ww, C.c_double), float(g_s), C.byref(opts),
                                   int(iters), out, 32, C.byref(n), _stream(stream))
    _check(s, "tb_autotune", False)
    return [{"panel": out[i].panel, "streams": out[i].streams, "cheb_cpt": out[i].cheb_cpt,
             "ctas_per_sm": out[i].ctas_per_sm, "rate": out[i].rate} for i in range(n.value)]


def tb_default_csc_opts(**kw) -> CscOpts:
    """tb_csc_opts with the library defaults, fields overridden by keyword."""
    o = CscOpts()
    load_library().tb_default_csc_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _numel(a) -> int:
    return int(a.numel()) if hasattr(a, "numel") else int(np.asarray(a).size)


def _in_ptr(a, n: int, keep: list):
    """Pointer to n doubles: a CUDA tensor in place, anything else as a
    contiguous float64 host copy (kept alive in ``keep``)."""
    if a is None:
        return C.c_void_p(0)
    if hasattr(a, "is_cuda") and a.is_cuda:
        if a.dtype.itemsize != 8 or not a.is_contiguous() or a.numel() != n:
            raise ValueError("expected a contiguous float64 CUDA tensor of %d elements" % n)
        return C.c_void_p(a.data_ptr())
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if arr.size != n:
        raise ValueError("expected %d elements, got %d" % (n, arr.size))
    keep.append(arr)
    return C.c_void_p(arr.ctypes.data)


def tb_csc_hamiltonian(h: Handle, gamma, dq, stream=None) -> None:
    """Set the handle's Hamiltonian to H0 + H^CSC(dq) (dq None: back to H0)."""
    keep = []
    n = h.n_atoms
    g = _in_ptr(gamma, n * n, keep) if dq is not None else C.c_void_p(0)
    s = load_library().tb_csc_hamiltonian(h.ptr, g, _in_ptr(dq, n, keep), _stream(stream))
    _check(s, "tb_csc_hamiltonian", False)


def tb_csc_loop(h: Handle, z, w, gamma, q_ref, g_s=2.0, dq_init=None, copts: CscOpts | None = None,
                opts: SolveOpts | None = None, q_out=None, dq_out=None, stream=None, allow_unconverged=False):
    """Self-consistent Mulliken charges (Eq. Hap-CSC, linear mixing); returns
    (q, dq, stats dict)."""
    import torch
    keep = []
    n = h.n_atoms
    zz = _complex_host(z)
    ww = _complex_host(w)
    K = len(zz) // 2
    if q_out is None:
        q_out = torch.empty((n,), dtype=torch.float64, device="cuda")
    if dq_out is None:
        dq_out = torch.empty((n,), dtype=torch.float64, device="cuda")
    copts = copts or tb_default_csc_opts()
    opts = opts or tb_default_opts()
    st = CscStats()
    s = load_library().tb_csc_loop(h.ptr, K, _ptr(zz, C.c_double), _ptr(ww, C.c_double), float(g_s),
                                   _in_ptr(gamma, n * n, keep), _in_ptr(q_ref, n, keep), _in_ptr(dq_init, n, keep),
                                   C.byref(copts), C.byref(opts), _out_ptr(q_out), _out_ptr(dq_out),
                                   C.byref(st), _stream(stream))
    _check(s, "tb_csc_loop", allow_unconverged)
    stats = {"status": tb_status_string(s), "iterations": st.iterations, "residual": st.residual,
             "outer_iterations": st.outer_iterations, "inner_iterations": st.inner_iterations,
             "seconds": st.seconds}
    return q_out, dq_out, stats


def tb_generalized_lanczos(h: Handle, j: int, n_steps: int, inner_tol=1e-13, stream=None):
    """Lanczos coefficients (a[n_steps], b[n_steps+1], norm) as numpy arrays."""
    a = np.zeros(n_steps)
    b = np.zeros(n_steps + 1)
    nrm = np.zeros(1)
    s = load_library().tb_generalized_lanczos(h.ptr, int(j), int(n_steps), float(inner_tol),
                                              C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data),
                                              C.c_void_p(nrm.ctypes.data), _stream(stream))
    _check(s, "tb_generalized_lanczos", False)
    return a, b, float(nrm[0])


def tb_lanczos_green(a, b, norm: float, z, out=None, stream=None):
    """G_jj(z_k) from Lanczos coefficients (continued fraction on the
    device); returns a complex128 array (numpy unless ``out`` is given)."""
    keep = []
    n = len(a)
    zz = _complex_host(z)
    K = len(zz) // 2
    if out is None:
        out = np.zeros(K, dtype=np.complex128)
    s = load_library().tb_lanczos_green(_in_ptr(a, n, keep), _in_ptr(b, n + 1, keep), float(norm), n, K,
                                        _ptr(zz, C.c_double), _out_ptr(out), _stream(stream))
    _check(s, "tb_lanczos_green", False)
    return out


def tb_generalized_lanczos_batch(h: Handle, cols, n_steps: int, opts: SolveOpts | None = None, stream=None):
    """Lanczos coefficients of R columns: (a [R, n_steps], b [R, n_steps+1],
    norm [R]) as numpy arrays."""
    cc = np.ascontiguousarray(cols, dtype=np.int32)
    R = len(cc)
    a = np.zeros((R, n_steps))
    b = np.zeros((R, n_steps + 1))
    nrm = np.zeros(R)
    opts = opts or tb_default_opts()
    s = load_library().tb_generalized_lanczos_batch(h.ptr, R, _ptr(cc, C.c_int32), int(n_steps), C.byref(opts),
                                                    C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data),
                                                    C.c_void_p(nrm.ctypes.data), _stream(stream))
    _check(s, "tb_generalized_lanczos_batch", False)
    return a, b, nrm


def tb_lanczos_green_batch(a, b, norm, z, out=None, stream=None):
    """G_r(z_k) for R Lanczos processes (a [R, n], b [R, n+1], norm [R]);
    returns complex128 [R, K] (numpy unless ``out`` is given)."""
    keep = []
    a = np.ascontiguousarray(a, dtype=np.float64)
    R, n = a.shape
    zz = _complex_host(z)
    K = len(zz) // 2
    if out is None:
        out = np.zeros((R, K), dtype=np.complex128)
    s = load_library().tb_lanczos_green_batch(R, _in_ptr(a, R * n, keep), _in_ptr(b, R * (n + 1), keep),
                                              _in_ptr(norm, R, keep), n, K, _ptr(zz, C.c_double), _out_ptr(out),
                                              _stream(stream))
    _check(s, "tb_lanczos_green_batch", False)
    return out


def tb_generalized_lanczos_noalloc(h: Handle, j: int, n_steps: int, inner_tol=1e-13, stream=None, out=None):
    """Allocation-free variant of tb_generalized_lanczos: the library takes
    its scratch from one fixed device array instead of allocating, for callers
    that cannot allocate GPU memory during the call.  ``out`` may hold
    preallocated (a, b, norm) host arrays or device tensors; returns them."""
    if out is None:
        out = (np.zeros(n_steps), np.zeros(n_steps + 1), np.zeros(1))
    a, b, nrm = out
    s = load_library().tb_generalized_lanczos_noalloc(h.ptr, int(j), int(n_steps), float(inner_tol),
                                                      _out_ptr(a), _out_ptr(b), _out_ptr(nrm), _stream(stream))
    _check(s, "tb_generalized_lanczos_noalloc", False)
    return a, b, nrm


def tb_measure_fma_peak(mode: int, stream=None) -> float:
    """Measured FMA throughput in TFLOP/s: mode 0 scalar FP32, 1 packed FP32,
    2 FP64."""
    v = C.c_double()
    _check(load_library().tb_measure_fma_peak(int(mode), C.byref(v), _stream(stream)), "tb_measure_fma_peak", False)
    return v.value


def tb_status_string(s: int) -> str:
    return load_library().tb_status_string(int(s)).decode()


def tb_launch_count() -> int:
    return int(load_library().tb_launch_count())


def tb_profile_enable(enable: bool = True) -> None:
    load_library().tb_profile_enable(1 if enable else 0)


def tb_profile_busy(kernel) -> float:
    """Busy milliseconds of a kernel class: the union of its launch
    intervals over all streams since profiling was enabled."""
    kid = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    ms = C.c_double()
    _check(load_library().tb_profile_busy(kid, C.byref(ms)), "tb_profile_busy", False)
    return ms.value


def tb_profile_read(kernel) -> tuple:
    """(launches, total_ms) of a kernel class (name or TB_K_* id)."""
    kid = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    n = C.c_int64()
    ms = C.c_double()
    _check(load_library().tb_profile_read(kid, C.byref(n), C.byref(ms)), "tb_profile_read", False)
    return int(n.value), float(ms.value)

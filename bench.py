"""Throughput benchmark of the generalized shifted COCG hot path on GB300.

Workload: Si diamond supercell of 4096 atoms (8x8x8 conventional cells,
a = 5.431 A, Gaussian displacements 0.05 A, seed 3), sp3 STO basis
(N = 16384 orbitals, ~17 4x4 blocks per block row), H by the ASED rule
(K = 1.75), 256 shifts z_k = E_k + 0.01i eV with E_k the Gauss-Legendre
nodes on [-20, 5] eV, Mulliken projection (a7).  One step = four panels
of P right-hand sides e_j (in flight together) run through ``iters`` outer
iterations of the whole hot path (seed SpMM, inner solve for S^-1 -- FP32
Chebyshev corrections inside FP64 refinement on the default mixed path --,
shift updates, seed switching, charge accumulation), started from
r_0 = e_j.  The full solve of this
workload needs ~10^4-10^5 outer iterations per column, so a step is a
fixed chunk of it; the metric is the rate shift*RHS*iterations/s.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank solves its own panel of columns (weak
scaling); no collective touches the data path, only the timing barrier and
the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "shift*RHS*iterations/s at 1e-8 residual"
UNIT = "shift*RHS*iterations/s"
CELLS = (8, 8, 8)
SEED = 3
K_SHIFTS = 256
# ALU peaks for the roofline of ALU-bound kernels: measured on the device
# by the library's FMA microbenchmark at the start of a run (tb_measure_fma_peak);
# these nominal figures stand only until then (or if it fails)
FP64_PEAK_TFLOPS = 1.25       # GB300 FP64 (vector and tensor), nominal
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32 FMA lanes x clock
ALU_PEAK_SOURCE = "nominal"


def measure_alu_peaks(P):
    """FP32 (best of scalar and packed FMA) and FP64 FMA throughput of this
    device, measured; they replace the nominal peaks for this run."""
    global FP32_PEAK_TFLOPS, FP64_PEAK_TFLOPS, ALU_PEAK_SOURCE
    try:
        f32 = P.tb_measure_fma_peak(0)
        f32p = P.tb_measure_fma_peak(1)
        f64 = P.tb_measure_fma_peak(2)
    except Exception as e:  # noqa: BLE001 -- keep the nominal figures, say why
        return {"source": "nominal", "error": str(e)}
    FP32_PEAK_TFLOPS = max(f32, f32p)
    FP64_PEAK_TFLOPS = f64
    ALU_PEAK_SOURCE = "measured (tb_measure_fma_peak)"
    return {"source": ALU_PEAK_SOURCE, "fp32_fma_tflops": f32, "fp32_packed_fma_tflops": f32p,
            "fp64_fma_tflops": f64}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--panel", type=int, default=0,
                    help="RHS per panel; 0 = the library autotuner (tb_autotune) picks panel width, panels in "
                         "flight and Chebyshev-step form")
    ap.add_argument("--iters", type=int, default=40, help="outer iterations per step")
    ap.add_argument("--panels-per-step", type=int, default=4,
                    help="panels of columns per step; the library keeps up to four panels of one system in flight")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--inner-tol", type=float, default=1e-12, help="relative accuracy of r' = S^-1 r (both precisions)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target length of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed",
                    help="mixed: FP32 Chebyshev corrections inside FP64 refinement (FP64-accurate); fp64: every product in FP64")
    ap.add_argument("--inner-method", choices=["chebyshev", "cg"], default="chebyshev",
                    help="mixed: FP32 corrections by Chebyshev steps (default) or by FP32 CG")
    ap.add_argument("--compare-steps", type=int, default=2,
                    help="timed steps of the other precision, reported beside the headline (0: skip)")
    ap.add_argument("--no-batch", action="store_true", help="skip the ragged-batch measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the band-energy gradient measurement")
    ap.add_argument("--no-lanczos", action="store_true", help="skip the batched Lanczos measurement")
    ap.add_argument("--large", action="store_true",
                    help="instead of the benchmark step: the 100 000-atom Si system (25x25x20 cells), Chebyshev-step "
                         "time and HBM fraction per panel width, mixed vs FP64 calls and their populations")
    ap.add_argument("--water-order", choices=["placement", "morton"], default="placement",
                    help="--batch-full: molecules in their placement order or sorted by the Morton key of the O position")
    ap.add_argument("--adjoint-full", action="store_true",
                    help="measure the band-energy adjoint and forces on the cracked 7680-atom Si slab instead")
    ap.add_argument("--adjoint-cells", type=int, default=10,
                    help="diamond cells per edge of the cracked slab of --adjoint-full (10: the 7680-atom workload)")
    ap.add_argument("--adjoint-profile", action="store_true",
                    help="with --adjoint-full: per-kernel device time of the band-energy call (library CUDA events)")
    ap.add_argument("--batch-full", action="store_true",
                    help="instead of the benchmark step: 64 liquid-water boxes of 512-1536 molecules (+H3O+) as one "
                         "ragged batch, 64 columns per box, 128 shifts, 20 outer iterations per call")
    ap.add_argument("--to-solution", type=int, default=32,
                    help="columns (one panel) run to the 1e-8 residual in every shift after the timed steps "
                         "(0: skip)")
    ap.add_argument("--csc-scf", type=int, default=1,
                    help="timed SCF iterations of the charge-self-consistency measurement (0: skip)")
    return ap.parse_args()


def workload():
    from tbinputs import si_system, gauss_legendre_grid
    s = si_system(CELLS, sigma=0.05, seed=SEED, cutoff=4.0)
    z, w = gauss_legendre_grid(K_SHIFTS, -20.0, 5.0, 0.01)
    return s, z, w


def csc_measure(P, prec, n_scf, panel):
    """Charge self-consistency (Eq. Hap-CSC) on liquid water, 256 neutral
    molecules (768 atoms, N = 1536 orbitals), Klopman-Ohno gamma, 64
    Gauss-Legendre nodes on [-60, -8] eV at a broadening of 2 eV, all 1536
    columns per SCF iteration, linear mixing 0.3: one untimed SCF iteration,
    then n_scf iterations timed with CUDA events (the loop is not run to
    self-consistency here)."""
    import torch
    from tbinputs import water_system, gauss_legendre_grid, klopman_ohno_gamma, valence_populations
    s = water_system(256, seed=4, excess_proton=False)
    z, w = gauss_legendre_grid(64, -60.0, -8.0, 2.0)
    gamma = torch.tensor(klopman_ohno_gamma(s), device="cuda")
    q_ref = torch.tensor(valence_populations(s), device="cuda")
    h = P.tb_create_system(s)
    opts = P.tb_default_opts(tol=1e-8, precision=prec, panel=panel)
    copts = P.tb_default_csc_opts(max_scf=1, mix=0.3, scf_tol=1e-12)
    P.tb_csc_loop(h, z, w, gamma, q_ref, copts=copts, opts=opts, allow_unconverged=True)   # warm-up
    copts = P.tb_default_csc_opts(max_scf=n_scf, mix=0.3, scf_tol=1e-12)
    P.tb_profile_enable(True)
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    q, dq, st = P.tb_csc_loop(h, z, w, gamma, q_ref, copts=copts, opts=opts, allow_unconverged=True)
    ev1.record(stream)
    ev1.synchronize()
    n_csc, ms_csc = P.tb_profile_read("csc")
    P.tb_profile_enable(False)
    ms = ev0.elapsed_time(ev1)
    return {"workload": "liquid water, 256 H2O (768 atoms, N=1536 sp/s orbitals), Klopman-Ohno gamma, "
                        "64 GL shifts on [-60,-8] eV + 2i eV, all 1536 columns per SCF iteration, mixing 0.3",
            "panel": panel,
            "n_atoms": s.n_atoms, "N": s.n_orb, "blocks": s.nb, "scf_iterations": st["iterations"],
            "ms_per_scf_iteration": ms / max(1, st["iterations"]),
            "csc_kernels_ms_per_iteration": ms_csc / max(1, st["iterations"]),
            "csc_kernel_launches": n_csc,
            "shift_rhs_iterations_per_s": 64 * st["outer_iterations"] / (ms / 1e3),
            "dq_residual": st["residual"]}


def batch_measure(P, prec, panel):
    """Ragged batch: 8 liquid-water boxes of 64-192 molecules (one H3O+ each,
    seeded sizes), 64 seeded columns per box, 64 Gauss-Legendre shifts on
    [-60, -8] eV + 2i eV, solved to 1e-8 as one block-diagonal batch handle
    and, for comparison, box by box (one handle and solve per box); both
    timed with CUDA events."""
    import torch
    from tbinputs import water_system, gauss_legendre_grid
    rng = np.random.default_rng(4)
    sizes = [int(n) for n in rng.integers(64, 193, size=8)]
    boxes = [water_system(n, seed=10 + i) for i, n in enumerate(sizes)]
    cols = [np.sort(np.random.default_rng(5 + i).choice(b.n_orb, 64, replace=False)).astype(np.int32)
            for i, b in enumerate(boxes)]
    z, w = gauss_legendre_grid(64, -60.0, -8.0, 2.0)
    opts = P.tb_default_opts(tol=1e-8, precision=prec, panel=panel)
    hb = P.tb_create_batch(boxes)
    hs = [P.tb_create_system(b) for b in boxes]
    all_cols = np.concatenate([c + hb.orb_off[i] for i, c in enumerate(cols)]).astype(np.int32)
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()                                   # warm-up
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        its = fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1e3, its

    t_b, it_b = timed(lambda: P.tb_mulliken_orbital(hb, z, w, all_cols, 2.0, opts=opts)[1]["outer_iterations"])
    t_s, it_s = timed(lambda: sum(P.tb_mulliken_orbital(h, z, w, c, 2.0, opts=opts)[1]["outer_iterations"]
                                  for h, c in zip(hs, cols)))
    return {"workload": "ragged batch: 8 water boxes of %s molecules (+H3O+), 64 columns each, 64 GL shifts "
                        "on [-60,-8] eV + 2i eV, tol 1e-8" % sizes,
            "n_atoms": int(hb.n_atoms), "N": int(hb.n_orb), "panel": panel,
            "batched_shift_rhs_iterations_per_s": 64 * it_b / t_b,
            "per_box_shift_rhs_iterations_per_s": 64 * it_s / t_s,
            "batched_s": t_b, "per_box_s": t_s, "speedup": t_s / t_b}


def adjoint_measure(P, prec, panel):
    """Band energy with dE/dH and dE/dS (every column of the system, its
    pattern rows projected with their z-derivatives) on Si 512 atoms (4x4x4
    cells, N = 2048, 68 pattern rows per column), 64 Gauss-Legendre shifts on
    [-20, 5] eV + 1i eV, tol 1e-8; timed with CUDA events."""
    import torch
    from tbinputs import si_system, gauss_legendre_grid
    s = si_system((4, 4, 4), sigma=0.05, seed=3)
    z, w = gauss_legendre_grid(64, -20.0, 5.0, 1.0)
    h = P.tb_create_system(s)
    opts = P.tb_default_opts(tol=1e-8, precision=prec, panel=panel)
    P.tb_band_energy(h, z, w, opts=opts, n_values=len(s.S_vals))        # warm-up
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    E, gH, gS, st = P.tb_band_energy(h, z, w, opts=opts, n_values=len(s.S_vals))
    ev1.record(stream)
    ev1.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    return {"workload": "band energy + dE/dH, dE/dS: Si 512 atoms (4x4x4 cells), N=2048, all columns, pattern "
                        "rows and z-derivatives projected, 64 GL shifts on [-20,5] eV + 1i eV, tol 1e-8",
            "n_atoms": s.n_atoms, "N": s.n_orb, "gradient_entries": len(s.S_vals), "panel": panel, "seconds": t,
            "shift_rhs_iterations_per_s": 64 * st["outer_iterations"] / t, "E_eV": E}


def lanczos_measure(P, s, prec, panel):
    """Generalized Lanczos (Section 3.2) for the LDOS of many orbitals: 1024
    seeded columns of the benchmark system as panels of ``panel`` columns,
    100 steps each, against the single-column call (FP64, as the paper's
    one-orbital use) on one of them; timed with CUDA events."""
    import torch
    cols = rank_columns(s.n_orb, 1024, 0, seed=7)
    h = P.tb_create_system(s)
    n_steps = 100
    opts = P.tb_default_opts(precision=prec, panel=panel, inner_tol=1e-12)
    stream = torch.cuda.current_stream()

    def timed(fn):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1e3

    P.tb_generalized_lanczos_batch(h, cols[:panel], 3, opts=opts)       # warm-up
    t_b = timed(lambda: P.tb_generalized_lanczos_batch(h, cols, n_steps, opts=opts))
    t_1 = timed(lambda: P.tb_generalized_lanczos(h, int(cols[0]), n_steps, inner_tol=1e-12))
    return {"workload": "generalized Lanczos, Si 4096 atoms, 1024 columns x 100 steps (panels of %d), "
                        "vs one column" % panel,
            "batched_s": t_b, "column_steps_per_s": 1024 * n_steps / t_b,
            "single_column_s": t_1, "single_column_steps_per_s": n_steps / t_1,
            "speedup_per_column": (1024 * n_steps / t_b) / (n_steps / t_1)}


def rank_columns(n_orb, panel, rank, seed=100):
    """Right-hand sides of one rank: a slice of one seeded permutation of all
    orbitals, so ranks never share a column (weak scaling by columns)."""
    perm = np.random.default_rng(seed).permutation(n_orb)
    lo = (rank * panel) % n_orb
    return np.sort(perm[lo:lo + panel]).astype(np.int32)


def reduce_max(value, world, device=None):
    """Max over ranks (timing only; no data-path collective)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def config_dict(args, s, precision=None):
    precision = precision or getattr(args, "precision", "fp64")
    return {
        "workload": (f"Si diamond {s.n_atoms} atoms ({CELLS[0]}x{CELLS[1]}x{CELLS[2]} cells), N={s.n_orb} sp3 "
                     f"orbitals, {K_SHIFTS} Gauss-Legendre shifts on [-20,5] eV + 0.01i eV, Mulliken projection, "
                     f"{args.iters} outer iterations per step"),
        "n_atoms": s.n_atoms, "N": s.n_orb, "blocks": int(s.nb), "shifts": K_SHIFTS, "panel": args.panel,
        "panels_per_step": args.panels_per_step,
        "iterations_per_step": args.iters, "tol": args.tol, "inner_tol": args.inner_tol,
        "precision": (("FP32 CG" if getattr(args, "inner_method", "chebyshev") == "cg" else "FP32 Chebyshev")
                      + " corrections (to 1e-6 per round) inside FP64 iterative refinement; FP64 outer SpMM, "
                      "vectors, recurrences, switching and charges" if precision == "mixed" else "FP64 throughout"),
        "l2": "flushed (256 MiB write) before every timed step", "seed": SEED,
        "basis": ("per-iteration rate over a fixed number of outer iterations from r_0 = e_j (tol 1e-8 is the "
                  "convergence test; no column converges within them); the rate to the 1e-8 residual is in "
                  "to_solution"),
    }


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(s, z, w, n_iter, col):
    """The oracle's method on one column for n_iter outer iterations (all
    shifts, Mulliken functional); returns seconds."""
    from oracle import dense, method
    Sc = s.to_csr()
    Hc = dense.ased_hamiltonian_sparse(Sc, s.eps, s.K, s.orbital_atom())
    F = Sc[col].toarray()
    c0 = time.process_time()
    t0 = time.perf_counter()
    method.generalized_shifted_cocg(Hc, Sc, z, col, tol=1e-8, inner_tol=1e-12, max_iter=n_iter, keep_full=False,
                                    functionals=F)
    t = time.perf_counter() - t0
    cores = max(1, math.ceil((time.process_time() - c0) / t - 0.05))
    return t, cores


def host_cpu_info():
    """Host cores and CPU model (lscpu, else /proc/cpuinfo)."""
    info = {"nproc": os.cpu_count()}
    try:
        info["affinity_cores"] = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        pass
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = dict(ln.split(":", 1) for ln in out.splitlines() if ":" in ln)
        model = " ".join(x.strip() for x in (fields.get("Vendor ID", ""), fields.get("Model name", "")) if x.strip())
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    info["model"] = model or "unknown"
    return info


_SINGLE = """
import os, sys, json
sys.path.insert(0, {root!r})
import bench
s, z, w = bench.workload()
t, c = bench.oracle_sample(s, z, w, {n}, 1234)
print(json.dumps({{"t": t, "cores": c}}))
"""


def cpu_baseline(s, z, w, target_s):
    """The oracle's method on one column of the workload, bounded to about
    target_s seconds: threaded (numpy / scipy as installed, all host cores)
    and, in a child process with the BLAS and OpenMP pools set to one
    thread, single-threaded on a shorter sample."""
    col = 1234
    t1, _ = oracle_sample(s, z, w, 2, col)
    per = t1 / 2.0
    n = int(max(2, min(400, target_s / max(per, 1e-6))))
    t, cores = oracle_sample(s, z, w, n, col)
    rec = {"value": K_SHIFTS * n / t, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": (f"oracle.method.generalized_shifted_cocg (numpy + scipy.sparse CSR, inner CG to 1e-12), "
                      f"1 column x {n} outer iterations x {K_SHIFTS} shifts of the same workload, {t:.1f} s"),
           "cores_basis": "process CPU time / wall time of the threaded sample",
           "host": host_cpu_info()}
    n1 = max(2, n // 3)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", _SINGLE.format(root=ROOT, n=n1)], env=env, capture_output=True,
                           text=True, timeout=max(120.0, 4 * target_s))
        one = json.loads(r.stdout.strip().splitlines()[-1])
        rec["single_thread"] = {"value": K_SHIFTS * n1 / one["t"], "unit": UNIT, "cores": 1,
                                "sample": f"1 column x {n1} outer iterations, {one['t']:.1f} s, BLAS/OpenMP pools "
                                          "of one thread"}
    except (OSError, subprocess.SubprocessError, ValueError, IndexError, KeyError) as e:
        rec["single_thread"] = {"error": str(e)}
    return rec


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    s, z, w = workload()
    n_iter = args.iters
    times = []
    cores = 1
    for i in range(args.warmup + args.steps):
        t, c = oracle_sample(s, z, w, n_iter, 1234 + i)
        if i >= args.warmup:
            times.append(t)
            cores = max(cores, c)
    tot = sum(times)
    value = K_SHIFTS * n_iter * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config_dict(args, s, precision="fp64"), panel=1, panels_per_step=1, iterations_per_step=n_iter,
                       precision="FP64 throughout (CPU oracle: numpy + scipy.sparse)", l2="not applicable (CPU)",
                       workload=config_dict(args, s)["workload"] + "; reference arm: CPU oracle, 1 column per step"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"1 column x {n_iter} outer iterations x {K_SHIFTS} shifts per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def kernel_source_sha256(kernel_file, kernel_name):
    """sha256 of the text of one kernel's definition (from ``__global__`` to
    its closing brace) in a file of the CUDA sources; None if not found."""
    src = open(os.path.join(ROOT, "paper_1002_1202_gb300", "csrc", kernel_file)).read()
    m = re.search(r"__global__[^;{]*?\b%s\s*\(" % re.escape(kernel_name), src)
    if not m:
        return None
    i = src.index("{", m.end())
    depth = 0
    for j in range(i, len(src)):
        if src[j] == "{":
            depth += 1
        elif src[j] == "}":
            depth -= 1
            if depth == 0:
                return hashlib.sha256(src[m.start():j + 1].encode()).hexdigest()
    return None


TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")


def stored_traffic(kernel_file, kernel_name, panel=None):
    """DRAM bytes per launch from a committed ncu summary, valid only while
    the text of the kernel it was taken from is unchanged and (for entries
    captured per panel width) for the panel width it was taken at."""
    path = TRAFFIC_PATH
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel_name)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    if kernel_source_sha256(kernel_file, kernel_name) != rec.get("kernel_sha256"):
        return None
    if "by_panel" in rec:
        return rec["by_panel"].get(str(panel))
    if "panel" in rec and panel is not None and rec["panel"] != panel:
        return None
    return rec.get("dram_bytes_per_launch")


KERNEL_INFO = {
    # name: (source file, kernel name, dtype bytes of matrix / vector elements, FP64?)
    "inner_spmv": ("k_inner_spmv", 8, 16, True),
    "outer_spmm": ("k_outer_spmm", 8, 16, True),
    "refine_residual": ("k_refine_residual", 8, 16, True),
    "inner32_spmv": ("k_inner32_spmv", 4, 8, False),
    "inner32_cheb": ("k_inner32_cheb4", 4, 8, False),
}


# columns per thread of the Chebyshev step that the autotuner chose (None:
# the library default)
CHEB_CPT = None


def cheb_kernel_name(panel, n_atoms):
    """The Chebyshev step's kernel, as the library picks it: the autotuner's
    choice, else TB_CHEB_CPT, else four columns per thread with packed FMAs
    from 16 columns per panel on and two below that."""
    env = os.environ.get("TB_CHEB_CPT")
    cpt = CHEB_CPT if CHEB_CPT else (int(env) if env else (4 if panel >= 16 else 2))
    if cpt == 2 or panel < 4:
        return "k_inner32_cheb"
    return "k_inner32_cheb4"


DF_INSTR_PER_MAC = 12   # FP32 instructions of one double-float multiply-add (exact product + two-sum)


def roofline_for(kname, ms, launches, s, panel, peaks, mixed=False, busy_ms=None):
    """Roofline of one SpMM-type kernel: algorithmic flops and bytes per
    launch over its CUDA-event time per launch.  With two panels in flight
    the launches of a kernel class overlap (and share the GPU), so the time
    per launch is the class's busy time (union of its launch intervals,
    ``busy_ms``) over its launches; the mean of the individual durations is
    reported beside it.  On the mixed path the FP64-accurate
    products of the outer SpMM and the refinement residual run in
    double-float FP32 arithmetic, DF_INSTR_PER_MAC FP32 instructions per
    FP64 multiply-add; they are rated against the FP32 issue peak (2 flop per
    FP32 lane-instruction), not against the FP64 units they do not use."""
    kern, mb, vb, fp64 = KERNEL_INFO[kname]
    if kname == "inner32_cheb":
        kern = cheb_kernel_name(panel, s.n_atoms)
    double_float = mixed and kname in ("outer_spmm", "refine_residual")
    nnz = 16 * s.nb
    mats = 2 if kname == "outer_spmm" else 1
    flops = 2.0 * nnz * 2 * panel * mats
    if kname == "inner32_cheb":
        flops += 5.0 * s.n_orb * 2 * panel      # d_{k+1} = d_{k-1} + omega (gamma (f - S d_k) + d_k - d_{k-1})
    # panel vectors moved once: the SpMVs read x and write y; the Chebyshev
    # step reads d_k, f and d_{k-1} and writes d_{k+1}
    vec_io = {"inner_spmv": 2, "inner32_spmv": 2, "inner32_cheb": 4, "refine_residual": 3, "outer_spmm": 5}[kname]
    nbytes = mats * nnz * mb + 4 * s.nb + 4 * (s.n_atoms + 1) + vec_io * s.n_orb * panel * vb
    mean_s = ms / max(launches, 1) / 1e3
    avg_s = busy_ms / max(launches, 1) / 1e3 if busy_ms else mean_s
    if avg_s <= 0:
        return None
    tf = flops / avg_s / 1e12
    gbs = nbytes / avg_s / 1e9
    if double_float:
        tf32 = flops / 2 * DF_INSTR_PER_MAC * 2 / avg_s / 1e12
        rec = {"bound": "alu", "achieved": tf32, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": tf32 / FP32_PEAK_TFLOPS, "fp64_equivalent_tflops": tf,
               "peak_source": "FP32 FMA peak (" + ALU_PEAK_SOURCE + "); double-float "
                              "products counted as 12 FP32 instructions per FP64 multiply-add"}
    elif fp64:
        rec = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": tf / FP64_PEAK_TFLOPS,
               "peak_source": "FP64 FMA peak (" + ALU_PEAK_SOURCE + ")"}
    else:
        f_alu = tf / FP32_PEAK_TFLOPS
        f_mem = gbs / peaks["hbm_gbs"]
        if f_mem >= f_alu:
            rec = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": f_mem,
                   "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)"}
        else:
            rec = {"bound": "alu", "achieved": tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": f_alu,
                   "peak_source": "FP32 FMA peak (" + ALU_PEAK_SOURCE + ")"}
    rec.update({"kernel": kern, "launches": launches, "avg_launch_us": avg_s * 1e6,
                "avg_launch_us_basis": "busy time (union of launch intervals on all streams) / launches",
                "mean_launch_duration_us": mean_s * 1e6,
                "flops_per_launch": flops, "algorithmic_bytes_per_launch": int(nbytes),
                "traffic": stored_traffic("tb_kernels.cu", kern, panel)})
    return rec


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except (OSError, ValueError, KeyError):
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1002_1202_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P.build()
    s, z, w = workload()
    h = P.tb_create_system(s)
    alu_peaks = measure_alu_peaks(P)
    prec = 1 if args.precision == "mixed" else 0
    inner_method = P.tb.TB_INNER_CG if args.inner_method == "cg" else P.tb.TB_INNER_CHEBYSHEV
    tune = None
    run_panel = args.panel
    if args.panel == 0:
        # the library's autotuner: panel width, panels in flight and the
        # Chebyshev-step form, 3 outer iterations per candidate; the best is
        # kept in the handle and used by the calls below (panel 0)
        o_t = P.tb_default_opts(tol=args.tol, precision=prec, inner_tol=args.inner_tol, inner_method=inner_method)
        tune = P.tb_autotune(h, z, w, 2.0, opts=o_t, iters=3)
        best = tune[0]["panel"]
        global CHEB_CPT
        CHEB_CPT = tune[0]["cheb_cpt"] or None
        if world > 1:
            t = torch.tensor([best], device="cuda", dtype=torch.int64)
            dist.broadcast(t, 0)
            best = int(t.item())
            run_panel = best       # ranks agree on one explicit width
        args.panel = best
    cols = rank_columns(s.n_orb, args.panel * args.panels_per_step, rank)
    ncols = len(cols)
    opts = P.tb_default_opts(max_iter=args.iters, panel=run_panel, tol=args.tol, precision=prec,
                             inner_tol=args.inner_tol, inner_method=inner_method)
    q_dev = torch.empty(ncols, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(out):
        return P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=opts, out=out, allow_unconverged=True)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(q_dev)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    P.tb_profile_enable(True)
    launches0 = P.tb_launch_count()
    times = []
    stats = []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, st = step(q_dev)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
        stats.append(st)
    barrier()
    launches = P.tb_launch_count() - launches0
    kernel_ms = {k: P.tb_profile_read(k) for k in P.tb.KERNELS}
    kernel_busy = {k: P.tb_profile_busy(k) for k in KERNEL_INFO}
    P.tb_profile_enable(False)
    clk = clocks.stop()
    total = reduce_max(sum(times), world, "cuda")
    units_per_step = K_SHIFTS * ncols * args.iters
    value = world * units_per_step * args.steps / total
    # active-shift variant: (column, shift) pairs not yet converged at each step
    act = 0
    for st in stats:
        ci = st["conv_iter"]
        act += int(np.sum(np.where(ci < 0, args.iters, np.minimum(ci, args.iters))))
    active_value = world * act / total

    # e2e: the same call with pinned host buffers (inputs copied in, charges read back)
    z_h = torch.from_numpy(np.ascontiguousarray(z)).pin_memory().numpy()
    w_h = torch.from_numpy(np.ascontiguousarray(w)).pin_memory().numpy()
    c_h = torch.from_numpy(np.ascontiguousarray(cols)).pin_memory().numpy()
    q_h = torch.empty(ncols, dtype=torch.float64).pin_memory().numpy()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        P.tb_mulliken_orbital(h, z_h, w_h, c_h, 2.0, opts=opts, out=q_h, allow_unconverged=True)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_tot = reduce_max(sum(e2e_times), world, "cuda")
    e2e = {"value": world * units_per_step * args.steps / e2e_tot, "unit": UNIT,
           "h2d_bytes_per_step": int(z_h.nbytes + w_h.nbytes + c_h.nbytes), "d2h_bytes_per_step": int(q_h.nbytes)}

    # roofline of the dominant kernel (largest device time in the timed region)
    peaks = measured_peaks()
    dom = max((k for k in KERNEL_INFO), key=lambda k: kernel_ms[k][1])
    roofline = roofline_for(dom, kernel_ms[dom][1], kernel_ms[dom][0], s, args.panel, peaks, prec == 1,
                            kernel_busy[dom])
    others = {k: roofline_for(k, kernel_ms[k][1], kernel_ms[k][0], s, args.panel, peaks, prec == 1, kernel_busy[k])
              for k in KERNEL_INFO if k != dom and kernel_ms[k][0] > 0}
    share = {k: round(v[1], 3) for k, v in kernel_ms.items() if v[0] > 0}
    # second part of the metric: SpMM algorithmic HBM GB/s against the measured copy peak
    spmm_hbm = {}
    for k in ("inner32_cheb", "inner32_spmv", "outer_spmm", "inner_spmv"):
        rec = roofline if roofline and roofline.get("kernel") == KERNEL_INFO[k][0] else others.get(k)
        if not rec:
            continue
        gbs = rec["algorithmic_bytes_per_launch"] / (rec["avg_launch_us"] * 1e-6) / 1e9
        spmm_hbm[k] = {"kernel": rec["kernel"], "algorithmic_GBps": gbs, "peak_GBps": peaks["hbm_gbs"],
                       "frac": gbs / peaks["hbm_gbs"],
                       "note": "algorithmic bytes (matrix once, every panel vector the kernel touches read or "
                               "written once) per busy time per launch; at 128-256 columns per panel the SpMM "
                               "does 8-16 flop per such byte, so it is limited by the gathers and the ALUs, not "
                               "by HBM"}

    # the other precision on the same panel, for comparison
    compare = None
    if args.compare_steps > 0:
        o2 = P.tb_default_opts(max_iter=args.iters, panel=args.panel, tol=args.tol, precision=1 - prec,
                               inner_tol=args.inner_tol)
        P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=o2, out=q_dev, allow_unconverged=True)
        ct = []
        for _ in range(args.compare_steps):
            flush.zero_()
            barrier()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=o2, out=q_dev, allow_unconverged=True)
            ev1.record(stream)
            ev1.synchronize()
            ct.append(ev0.elapsed_time(ev1) / 1e3)
        ctot = reduce_max(sum(ct), world, "cuda")
        compare = {"precision": "fp64" if prec == 1 else "mixed", "steps": args.compare_steps,
                   "value": world * units_per_step * args.compare_steps / ctot,
                   "ms_per_step": 1e3 * ctot / args.compare_steps}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32" if prec else "f64", "data": "synthetic",
        "config": config_dict(args, s), "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
        "roofline": roofline, "roofline_other_kernels": others, "active_shift_value": active_value,
        "kernel_ms": share, "spmm_hbm": spmm_hbm, "other_precision": compare, "peaks": dict(peaks, alu=alu_peaks),
        "autotune": tune,
        "inner_redos": sum(st["inner_redos"] for st in stats),
        "inner_iterations_per_outer": (sum(st["inner_iterations"] for st in stats)
                                       / max(1, sum(st["max_column_iterations"] + 1 for st in stats))),
    }
    if world == 1 and not args.no_lanczos:
        line["lanczos"] = lanczos_measure(P, s, prec, args.panel)
    if world == 1 and not args.no_adjoint:
        line["adjoint"] = adjoint_measure(P, prec, args.panel)
    if world == 1 and not args.no_batch:
        line["batch"] = batch_measure(P, prec, args.panel)
    if world == 1 and args.csc_scf > 0:
        line["csc"] = csc_measure(P, prec, args.csc_scf, args.panel)
    if world == 1 and args.to_solution > 0:
        line["to_solution"] = to_solution_measure(P, h, s, z, w, prec, inner_method, n_cols=args.to_solution)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(s, z, w, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def to_solution_measure(P, h, s, z, w, prec, inner_method, n_cols=4, max_iter=100000):
    """n_cols seeded columns of the benchmark workload run until every one of
    the K shifts meets the 1e-8 residual (one panel, Mulliken projection, the
    benchmark's precision and inner tolerance): outer iterations to
    convergence per column, wall time, and shift*RHS*iterations/s with
    n_j = the iterations column j ran (all K shifts counted until the
    column's last converges) and with only the unconverged shifts counted.
    The true residuals of such solutions are checked against the dense
    definition by the GPU test of the same configuration."""
    import torch
    cols = rank_columns(s.n_orb, n_cols, 0, seed=77)
    opts = P.tb_default_opts(max_iter=max_iter, panel=n_cols, tol=1e-8, precision=prec, inner_tol=1e-12,
                             inner_method=inner_method)
    P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=P.tb_default_opts(max_iter=3, panel=n_cols, precision=prec),
                          allow_unconverged=True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    _, st = P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=opts, allow_unconverged=True)
    ev1.record()
    ev1.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    ci = np.asarray(st["conv_iter"]).reshape(n_cols, -1)
    K = ci.shape[1]
    per_col = [int(r.max()) + 1 if np.all(r >= 0) else max_iter for r in ci]
    return {"workload": "%d seeded columns of the benchmark system to the 1e-8 residual in every one of %d shifts, "
                        "one panel" % (n_cols, K),
            "status": st["status"], "all_converged": bool(np.all(ci >= 0)), "seconds": t,
            "outer_iterations_per_column": per_col,
            "value": K * sum(per_col) / t, "unit": UNIT,
            "active_shift_value": float(np.sum(np.where(ci >= 0, ci + 1, max_iter))) / t}


def run_adjoint_full(args):
    """The differentiation workload at its stated size: the cracked Si slab
    (10 x 10 x 10 cells, 7680 atoms, N = 30720), 128 Gauss-Legendre shifts on
    [-20, 5] eV + 1i eV (the workload names the shift count, not the
    broadening), mixed precision: the band energy with dE/dH and dE/dS at
    every stored entry (all columns, their pattern rows projected with the
    z-derivatives), chained to per-atom forces through the overlap's bond
    derivatives (Eq. Hap-1 for H).  Timed with CUDA events; one JSON line."""
    import torch
    from tbinputs import si_slab_system, gauss_legendre_grid, overlap_bond_derivatives
    P = __import__("paper_1002_1202_gb300")
    P.build()
    t0 = time.time()
    c = args.adjoint_cells
    s = si_slab_system(cells=(c, c, c))
    dS = overlap_bond_derivatives(s)
    build_s = time.time() - t0
    print("slab %d atoms, N=%d, %d blocks built in %.1f s" % (s.n_atoms, s.n_orb, s.nb, build_s),
          file=sys.stderr, flush=True)
    z, w = gauss_legendre_grid(128, -20.0, 5.0, 1.0)
    h = P.tb_create_system(s)
    opts = P.tb_default_opts(tol=1e-8, precision=1)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    if args.adjoint_profile:
        P.tb_profile_enable(True)
    torch.cuda.synchronize()
    ev[0].record(stream)
    E, gH, gS, st = P.tb_band_energy(h, z, w, opts=opts, n_values=len(s.S_vals))
    ev[1].record(stream)
    F = P.tb_forces(h, gH, gS, dS)
    ev[2].record(stream)
    ev[2].synchronize()
    kernel_ms = None
    if args.adjoint_profile:
        kernel_ms = {k: [v[0], round(v[1], 3)] for k, v in ((k, P.tb_profile_read(k)) for k in P.tb.KERNELS)
                     if v[0] > 0}
        P.tb_profile_enable(False)
    F = np.asarray(F.cpu().numpy() if hasattr(F, "cpu") else F)
    t_e = ev[0].elapsed_time(ev[1]) / 1e3
    print(json.dumps({
        "metric": "adjoint_full", "unit": UNIT,
        "workload": "cracked Si slab %dx%dx%d cells, %d atoms, N=%d, %d blocks; 128 GL shifts on [-20,5] eV + 1i eV; "
                    "band energy, dE/dH and dE/dS at every stored entry, forces; mixed precision" % (
                        c, c, c, s.n_atoms, s.n_orb, s.nb),
        "host_build_s": build_s, "band_energy_s": t_e, "forces_ms": ev[1].elapsed_time(ev[2]),
        "status": st["status"], "E_eV": E, "outer_iterations": st["outer_iterations"],
        "value": 128 * st["outer_iterations"] / t_e, "gradient_entries": int(len(s.S_vals)),
        "net_force_over_max": float(np.abs(F.sum(axis=0)).max() / max(np.abs(F).max(), 1e-300)),
        "kernel_launches_ms": kernel_ms}))
    return 0


def run_large(args):
    """The 100 000-atom Si system (25x25x20 diamond cells, seed 6, N = 400 000,
    1.68 M blocks; its FP32 S, 108 MB, exceeds L2): for panels of 4 ... 128
    columns, one Mulliken call of 3 outer iterations (after a warm-up call)
    with the library's per-launch CUDA events on, giving the Chebyshev step's
    busy time per launch and its algorithmic bytes (FP32 S once, index arrays
    once, four panel passes) against the measured HBM copy rate; at 32 and
    128 columns the same call in FP64, and the largest difference of the two
    precisions' populations.  One JSON line."""
    import torch
    from tbinputs import si_system, gauss_legendre_grid
    P = __import__("paper_1002_1202_gb300")
    P.build()
    t0 = time.time()
    s = si_system((25, 25, 20), seed=6)
    build_s = time.time() - t0
    z, w = gauss_legendre_grid(128, -20.0, 5.0, 0.01)
    h = P.tb_create_system(s)
    peaks = measured_peaks()
    nnz = 16 * s.nb
    rows = []
    for panel in (4, 8, 16, 32, 64, 128):
        cols = rank_columns(s.n_orb, panel, 0)
        rec = {"panel": panel}
        q = {}
        for prec in ((1, 0) if panel in (32, 128) else (1,)):
            opts = P.tb_default_opts(max_iter=3, panel=panel, precision=prec, tol=1e-8, inner_tol=1e-12)
            P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=opts, allow_unconverged=True)
            torch.cuda.synchronize()
            P.tb_profile_enable(True)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            out, _ = P.tb_mulliken_orbital(h, z, w, cols, 2.0, opts=opts, allow_unconverged=True)
            ev1.record()
            ev1.synchronize()
            q[prec] = out.cpu().numpy()
            if prec == 1:
                n_l, _ms = P.tb_profile_read("inner32_cheb")
                busy = P.tb_profile_busy("inner32_cheb")
                us = busy / max(n_l, 1) * 1e3
                nbytes = nnz * 4 + 4 * s.nb + 4 * (s.n_atoms + 1) + 4 * s.n_orb * panel * 8
                rec.update({"cheb_launches": n_l, "cheb_us_per_launch": us,
                            "cheb_algorithmic_GBps": nbytes / us / 1e3,
                            "cheb_hbm_frac": nbytes / us / 1e3 / peaks["hbm_gbs"]})
                rec["mixed_call_ms"] = ev0.elapsed_time(ev1)
            else:
                rec["fp64_call_ms"] = ev0.elapsed_time(ev1)
            P.tb_profile_enable(False)
        if 0 in q:
            rec["max_population_difference"] = float(np.abs(q[1] - q[0]).max())
            rec["fp64_over_mixed_time"] = rec["fp64_call_ms"] / rec["mixed_call_ms"]
        rows.append(rec)
    print(json.dumps({"metric": "large_system", "workload": "Si diamond 25x25x20 cells, 100000 atoms, N=400000, "
                      "%d blocks, 128 Gauss-Legendre shifts on [-20,5] eV + 0.01i eV, 3 outer iterations per call, "
                      "mixed precision (FP32 Chebyshev corrections) and FP64" % s.nb,
                      "build_s": build_s, "peaks": peaks, "panels": rows}))
    return 0


def _water_box(args):
    from tbinputs import water_system
    n, seed, order = args
    return water_system(n, seed=seed, order=order)


def run_batch_full(args):
    """The ragged-batch workload at its stated size: 64 seeded liquid-water
    boxes of 512-1536 molecules (one H3O+ each; sizes from
    default_rng(4)), built on the host cores by a spawned process pool
    before the first CUDA call, created as one batch handle; 64 seeded
    columns per box (4096 in all), 128 Gauss-Legendre shifts on
    [-20, 5] eV + 0.01i eV, mixed precision, 20 outer iterations per call
    (the full solve needs thousands).  Timed with CUDA events over two calls
    after a warm-up; beside it the same columns box by box for the first
    8 boxes.  One JSON line."""
    import multiprocessing as mp
    sizes = [int(n) for n in np.random.default_rng(4).integers(512, 1537, size=64)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        boxes = pool.map(_water_box, [(n, 1000 + i, args.water_order) for i, n in enumerate(sizes)])
    build_s = time.time() - t0
    import torch
    from tbinputs import gauss_legendre_grid
    P = __import__("paper_1002_1202_gb300")
    P.build()
    hb = P.tb_create_batch(boxes)
    cols = [np.sort(np.random.default_rng(5 + i).choice(b.n_orb, 64, replace=False)).astype(np.int32)
            for i, b in enumerate(boxes)]
    all_cols = np.concatenate([c + hb.orb_off[i] for i, c in enumerate(cols)]).astype(np.int32)
    z, w = gauss_legendre_grid(128, -20.0, 5.0, 0.01)
    iters = 20
    opts = P.tb_default_opts(max_iter=iters, panel=64, precision=1, tol=1e-8, inner_tol=1e-12)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / reps

    t_b = timed(lambda: P.tb_mulliken_orbital(hb, z, w, all_cols, 2.0, opts=opts, allow_unconverged=True), 2)
    hs = [P.tb_create_system(b) for b in boxes[:8]]
    t_s = timed(lambda: [P.tb_mulliken_orbital(h, z, w, c, 2.0, opts=opts, allow_unconverged=True)
                         for h, c in zip(hs, cols[:8])], 1)
    units = 128 * len(all_cols) * iters
    print(json.dumps({
        "metric": "batch_full", "unit": UNIT,
        "workload": "64 water boxes of %d-%d molecules (+H3O+), %d orbitals in all, 64 columns per box, 128 "
                    "Gauss-Legendre shifts on [-20,5] eV + 0.01i eV, %d outer iterations per call, mixed precision; "
                    "molecules in %s order" % (min(sizes), max(sizes), int(hb.n_orb), iters, args.water_order),
        "build_s": build_s, "batched_s": t_b, "value": units / t_b,
        "per_box_first8_s": t_s, "per_box_first8_value": 128 * 64 * 8 * iters / t_s,
        "sizes": sizes}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.large:
        return run_large(args)
    if args.batch_full:
        return run_batch_full(args)
    if args.adjoint_full:
        return run_adjoint_full(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Host-side arithmetic of bench.py on CPU: the roofline record of a kernel
from its launch count and times, the kernel-text hash that guards stored
ncu traffic, and the per-panel-width traffic lookup."""
import types

import pytest

import bench


def _fake_system(n_atoms=4096, nb=69024):
    return types.SimpleNamespace(n_atoms=n_atoms, nb=nb, n_orb=4 * n_atoms)


def test_kernel_hash_covers_the_kernel_text():
    h = bench.kernel_source_sha256("tb_kernels.cu", "k_inner32_cheb4")
    assert h is not None and len(h) == 64
    assert bench.kernel_source_sha256("tb_kernels.cu", "k_inner32_cheb4") == h
    assert bench.kernel_source_sha256("tb_kernels.cu", "k_no_such_kernel") is None
    assert h != bench.kernel_source_sha256("tb_kernels.cu", "k_inner32_cheb")


def test_stored_traffic_is_per_panel_and_hash_guarded(monkeypatch, tmp_path):
    import json
    rec = {"k_inner32_cheb": {"kernel_sha256": bench.kernel_source_sha256("tb_kernels.cu", "k_inner32_cheb"),
                           "by_panel": {"128": 60e6, "256": 120e6}},
           "k_inner32_spmv": {"kernel_sha256": bench.kernel_source_sha256("tb_kernels.cu", "k_inner32_spmv"),
                              "dram_bytes_per_launch": 42e6, "panel": 256}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(path))
    t128 = bench.stored_traffic("tb_kernels.cu", "k_inner32_cheb", 128)
    t256 = bench.stored_traffic("tb_kernels.cu", "k_inner32_cheb", 256)
    assert t128 == 60e6 and t256 == 120e6
    assert bench.stored_traffic("tb_kernels.cu", "k_inner32_cheb", 64) is None
    # an entry captured at one width is not reported for another
    assert bench.stored_traffic("tb_kernels.cu", "k_inner32_spmv", 128) is None
    assert bench.stored_traffic("tb_kernels.cu", "k_inner32_spmv", 256) == 42e6
    # once the kernel text changes the stored figure is void
    monkeypatch.setattr(bench, "kernel_source_sha256", lambda f, k: "0" * 64)
    assert bench.stored_traffic("tb_kernels.cu", "k_inner32_cheb", 128) is None


def test_committed_traffic_entries_match_their_kernels():
    """Every entry of the committed traffic record names a kernel that
    exists; an entry whose kernel text changed is reported as void (None)
    rather than carried over."""
    import json
    import os
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for name in rec:
        assert bench.kernel_source_sha256("tb_kernels.cu", name) is not None, name


@pytest.mark.parametrize("panel", [128, 256])
def test_roofline_of_the_chebyshev_step(panel):
    s = _fake_system()
    peaks = {"hbm_gbs": 6778.7}
    launches, busy_ms = 1000, 40.0 * panel / 128          # 40 us per launch at P = 128
    rec = bench.roofline_for("inner32_cheb", 4 * busy_ms, launches, s, panel, peaks, True, busy_ms)
    nnz = 16 * s.nb
    flops = 2.0 * nnz * 2 * panel + 5.0 * s.n_orb * 2 * panel
    nbytes = nnz * 4 + 4 * s.nb + 4 * (s.n_atoms + 1) + 4 * s.n_orb * panel * 8
    avg_s = busy_ms / launches / 1e3
    assert rec["kernel"] == "k_inner32_cheb4"
    assert rec["flops_per_launch"] == pytest.approx(flops)
    assert rec["algorithmic_bytes_per_launch"] == int(nbytes)
    assert rec["avg_launch_us"] == pytest.approx(avg_s * 1e6)
    assert rec["mean_launch_duration_us"] == pytest.approx(4 * avg_s * 1e6)
    f_mem = nbytes / avg_s / 1e9 / peaks["hbm_gbs"]
    f_alu = flops / avg_s / 1e12 / bench.FP32_PEAK_TFLOPS
    assert rec["frac"] == pytest.approx(max(f_mem, f_alu))
    assert rec["bound"] == ("hbm" if f_mem >= f_alu else "alu")
    assert rec["achieved"] / rec["peak"] == pytest.approx(rec["frac"])


def test_roofline_of_double_float_kernels_counts_fp32_instructions():
    s = _fake_system()
    rec = bench.roofline_for("refine_residual", 10.0, 100, s, 128, {"hbm_gbs": 6778.7}, True, 10.0)
    flops = 2.0 * 16 * s.nb * 2 * 128
    avg_s = 10.0 / 100 / 1e3
    assert rec["bound"] == "alu" and rec["unit"] == "TFLOP/s"
    assert rec["achieved"] == pytest.approx(flops / 2 * bench.DF_INSTR_PER_MAC * 2 / avg_s / 1e12)
    assert rec["fp64_equivalent_tflops"] == pytest.approx(flops / avg_s / 1e12)

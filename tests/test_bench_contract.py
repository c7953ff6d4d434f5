"""The benchmark's reference arm (the FP64 oracle timed on the host) and its
JSON line, on the CPU: one small run through bench.py's own entry point."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "64", "--J", "4",
                          "--steps", "3", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_reference_arm_non_zero_rank_is_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "64", "--J", "4",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT,
                         env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


def test_direct_map_tap_count_and_alu_peak():
    """The direct M_ap roofline counts the lattice offsets 0 < |d| <= R
    (brute force here) and derives the FP32 FMA peak from unit counts."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    for R in (1.0, 2.0, 3.5, 16.0, 64.0):
        Ri = int(np.floor(R))
        d = np.arange(-Ri, Ri + 1)
        r2 = d[:, None] ** 2 + d[None, :] ** 2
        assert bench.disc_taps(R) == int(((r2 > 0) & (r2 <= R * R)).sum())
    assert abs(bench.FP32_PEAK_TFLOPS - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert bench.algo_bytes_per_px_launch("starlet_tile", 2) == 16
    assert bench.algo_bytes_per_px_launch("starlet_col", 2) == 16 and bench.algo_bytes_per_px_launch("starlet_row", 3) == 8
    assert bench.algo_bytes_per_px_launch("starlet_col", 2, one_pass=True) == 12


def test_roofline_uses_the_method_bytes():
    """The bench's roofline credits the method's bytes: a large scale is 12
    B/px (read c_{j-1}, write c_j and w_j) over its row and column launches
    together, KS 12 B/px over its three passes, the step 12 + 4 (J + 1) B/px
    over the step time, the HBM floor 8 + 4J (shear in, J arrays out)."""
    sys.path.insert(0, ROOT)
    import bench
    px = 32 * 1024 * 1024
    per_kind = {"fft_rows_fwd": (0.22, 8), "fft_cols_ks": (0.22, 8), "fft_rows_inv": (0.12, 8),
                "starlet_tile": (0.18, 8), "starlet_row": (0.39, 32), "starlet_col": (0.39, 32)}
    r = bench.step_roofline(per_kind, px, 7, 2, 0.8, 6800.0, "measured")
    assert r["kernel"].startswith("starlet_large_scale")
    pair_ms = (0.39 + 0.39) / 32  # one scale of one 4-map chunk
    assert abs(r["achieved"] - 12 * px / 8 / (pair_ms * 1e-3) / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6800.0) < 1e-12
    assert abs(r["step"]["frac"] - 44 * px / 0.8e-3 / 1e9 / 6800.0) < 1e-12
    assert abs(r["step"]["floor_frac"] - 36 * px / 0.8e-3 / 1e9 / 6800.0) < 1e-12
    ks = r["groups"]["ks"]
    assert abs(ks["achieved_gbs"] - 12 * px / 8 / ((0.56 / 8) * 1e-3) / 1e9) < 1e-6
    assert r["groups"]["starlet_tile"]["method_bytes_per_px"] == 16


def test_roofline_one_pass_scales_take_the_dominant_kernel():
    """With one pass per large scale the kernel with the most device time
    (here the one-pass scale kernel, 0.48 ms) sets the roofline, even when
    the three KS passes together take longer."""
    sys.path.insert(0, ROOT)
    import bench
    px = 32 * 1024 * 1024
    per_kind = {"fft_rows_fwd": (0.22, 8), "fft_cols_ks": (0.22, 8), "fft_rows_inv": (0.12, 8),
                "starlet_tile": (0.19, 8), "starlet_col": (0.48, 32)}
    r = bench.step_roofline(per_kind, px, 7, 2, 0.7, 6800.0, "measured")
    assert r["dominant_kernel"] == "starlet_col" and r["kernel"].startswith("starlet_large_scale")
    assert abs(r["achieved"] - 12 * px / 8 / ((0.48 / 32) * 1e-3) / 1e9) < 1e-6
    assert r["kernel_bytes_per_launch"] == 12 * px / 8


def test_roofline_real_output_ks_kernel_bytes():
    """With the real-output KS inverse (the default from 512^2 up) the three
    KS passes move 16 + 12 + 8 = 36 B/px (the column pass writes, and the
    row inverse reads, the half spectrum) against 44 for the complex
    inverse; the method bytes credited to the group stay 12 B/px."""
    sys.path.insert(0, ROOT)
    import bench
    kinds = ("fft_rows_fwd", "fft_cols_ks", "fft_rows_inv")
    assert [bench.algo_bytes_per_px_launch(k, 2, ks_real=True) for k in kinds] == [16, 12, 8]
    assert [bench.algo_bytes_per_px_launch(k, 2, ks_real=False) for k in kinds] == [16, 16, 12]
    px = 32 * 1024 * 1024
    per_kind = {"fft_rows_fwd": (0.175, 8), "fft_cols_ks": (0.183, 8), "fft_rows_inv": (0.102, 8),
                "starlet_tile": (0.167, 8), "starlet_col": (0.436, 32)}
    r = bench.step_roofline(per_kind, px, 7, 2, 0.572, 6776.6, "measured", ks_real=True)
    ks = r["groups"]["ks"]
    assert ks["method_bytes_per_px"] == 12 and ks["kernel_bytes_per_launch"] == 36 * px / 8
    assert abs(r["step"]["frac"] - 44 * px / 0.572e-3 / 1e9 / 6776.6) < 1e-12

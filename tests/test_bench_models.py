"""Host logic of bench.py: the algorithmic byte and flop models behind the
roofline objects, and the reference arm's JSON line (the oracle timed on the
host cores)."""
import json
import math
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_byte_model_at_256_fp32():
    """Per-launch algorithmic bytes at N = 256, P = 384, complex64: the arrays
    each pass must read and write once (unit N^2 h complex)."""
    N, P, h, esz = 256, 384, 128, 8
    kb = bench.kernel_bytes(N, P, esz, 1)
    U, A, Bq, Cq, Dq = 3 * N * N * h, 3 * P * N * h, 3 * P * P * h, 6 * P * P * h, 6 * P * N * h
    assert kb["inverse_y"] == (A + Bq) * esz
    assert kb["zpass"] == (Bq + Cq) * esz
    assert kb["forward_y"] == (Cq + Dq) * esz
    assert kb["fused_x"] == (Dq + U + U + 2 * U / 3 + A) * esz
    # the figures quoted with the rooflines
    assert round(kb["zpass"] / 1e9, 3) == 1.359
    assert round(kb["inverse_y"] / 1e9, 3) == 0.755
    assert round(kb["forward_y"] / 1e9, 3) == 1.510
    assert round(kb["fused_x"] / 1e9, 3) == 1.443
    # members scale every kind
    kb2 = bench.kernel_bytes(N, P, esz, 2)
    assert all(kb2[k] == 2 * kb[k] for k in kb)


def test_flop_model_and_fp64_peak():
    # 256^3: 1,400,832 complex lines of length 384 per right-hand side
    lines = 3 * 256 * 128 + 3 * 384 * 128 + 4.5 * 384 * 384 + 6 * 384 * 128 + 6 * 256 * 128
    assert lines == 1400832
    f = bench.fft_flops_per_step(256, 384)
    assert abs(f - 3 * lines * 5 * 384 * math.log2(384)) < 1.0
    assert round(f / 1e9, 1) == 69.3
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-12      # 152 SMs x 4 flops x 2.07 GHz


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["sample"]
    e = line["e2e"]
    assert e["value"] == line["value"] and e["unit"] == line["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # the line names the workload it actually times (a 16^3 sample of the main one)
    assert line["config"]["N"] == 16 and line["config"]["sample_of_N"] == 256
    assert "16^3" in line["config"]["workload"]
    assert cb["nproc"] >= 1


def test_cpu_baseline_all_cores_pool():
    """The all-core leg of the CPU baseline: one spawn-started single-threaded
    process per worker, each advancing its own member; a small case here."""
    sec = bench.oracle_all_cores(8, 2)
    assert 0 < sec < 120
    model, n = bench.host_cpu()
    assert n >= 1


def test_traffic_entry_names_its_capture():
    b, src = bench.traffic_entry("zpass", 256, "f32", 1)
    assert (b is None) == (src is None)
    if src is not None:
        assert os.path.exists(os.path.join(ROOT, src))
    assert bench.traffic_entry("zpass", 999, "f32", 1) == (None, None)


def test_fp64_roofline_model():
    """FP64 lines: the flop model times the double-single cost per flop (a sum
    11 FP32 operations, a product 7, two sums per product) against the FP32
    pipe (152 SMs x 128 lanes x 2.07 GHz)."""
    assert abs(bench.FP32_OPS_PEAK_T - 40.27392) < 1e-9
    assert abs(bench.DF64_OPS_PER_FLOP - 29.0 / 3.0) < 1e-15
    r = bench.fp64_roofline(256, 384, 60.0)
    f = bench.fft_flops_per_step(256, 384)
    assert abs(r["achieved"] - f * 29 / 3 / 0.06 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 40.27392) < 1e-15
    assert abs(r["fp64_equivalent_TFLOPs"] - f / 0.06 / 1e12) < 1e-12


def test_window_sizes_cover_the_timed_steps():
    """The timed region's windows: five of at least 20 steps where there are
    enough, fewer otherwise, one for short runs; they sum to the step count."""
    assert bench.window_sizes(300) == [60] * 5
    assert bench.window_sizes(101) == [21, 20, 20, 20, 20]
    assert bench.window_sizes(99) == [25, 25, 25, 24]
    assert bench.window_sizes(30) == [30] and bench.window_sizes(1) == [1]
    for k in range(1, 400):
        w = bench.window_sizes(k)
        assert sum(w) == k and (len(w) == 1 or min(w) >= 20) and len(w) <= 5

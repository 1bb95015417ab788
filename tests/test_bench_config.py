"""bench.py's workload table and options, on the CPU: every workload has a
loader or its own path, sampled-accuracy workloads are in the table, the
error-estimate factor defaults to 8 ulps, and the reference arm answers for
the batched workload without running anything."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workload_table():
    assert set(bench.ACCURACY_SAMPLE) <= set(bench.WORKLOADS)
    assert bench.WORKLOADS["pseudo_1e6"][1] and not bench.WORKLOADS["direct_8m"][1]
    src = open(os.path.join(ROOT, "bench.py")).read()
    for name in bench.WORKLOADS:
        assert f'"{name}"' in src.split("def load_workload")[1] or name in ("sphere_1e5", "batched_64"), name


def test_defaults(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.workload, a.precision, a.err_ulps, a.workers) == (1, "pseudo_1e6", "mixed", 0, 8)
    assert a.warmup >= 3 and a.h_tol == 1e-13
    assert bench.err_ulps(a) == 8
    a.err_ulps = 24
    assert bench.err_ulps(a) == 24


def test_reference_arm_batched_is_unavailable():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "batched_64"], capture_output=True, text=True, check=True, cwd=ROOT)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_roofline_follows_the_counted_work_and_measured_peaks():
    """achieved = the oracle-counted work per pair x pairs / time, against the
    measured peak of the executing pipe; nominal figures only beside it."""
    peaks = dict(fp32_tflops=70.0, fp64_tflops=1.1, xu_tops=4.5, sm_count=152, sm_clock_mhz=2070.0)
    r = bench.roofline(24_000_000, 120.0, "mixed", "pseudo_1e6", peaks, 2070.0)
    aw = bench.ALGO_WORK["pseudo_1e6"]
    assert abs(r["achieved"] - 24e6 * aw["flops"] / 0.12 / 1e12) < 1e-9
    assert r["peak"] == 70.0 and abs(r["frac"] - r["achieved"] / 70.0) < 1e-12
    assert r["pipe"] == "fp32" and r["nominal_peak"] > r["peak"]
    assert abs(r["sfu"]["achieved"] - 24e6 * (aw["sqrt"] + aw["transcendental"]) / 0.12 / 1e12) < 1e-9
    assert "implementation" in r
    r64 = bench.roofline(24_000_000, 4000.0, "fp64", "pseudo_1e6", peaks, None)
    assert r64["peak"] == 1.1 and r64["kernel"] == "k_map_fp64" and "implementation" not in r64
    assert bench.roofline(1, 1.0, "mixed", "full_8m", peaks) is None

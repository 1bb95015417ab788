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

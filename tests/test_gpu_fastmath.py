"""The FP32 pass's own e^x - 1 and square root (csrc/quad32.cuh: ex_m1,
sqrt_nr) against a double-precision reference on dense samples of their
ranges, beside CUDA's expm1f and sqrtf on the same inputs: ex_m1 within 2
ulp, sqrt_nr within 1 ulp, subnormals and 0 included.  The integer
double -> float-float split of the derived geometry and the h-solver's
conversions to and from float (csrc/split.cuh) equal, bit for bit, to the
conversions they replace, ties and carries included."""
import os
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ex_m1_and_sqrt_nr_accuracy():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "fastmath")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-I", os.path.join(ROOT, "paper_2410_15227_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "gpu_fastmath_check.cu"), "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    res = {p[0]: (float(p[1]), float(p[2]), int(p[3])) for p in (line.split() for line in out.strip().splitlines())}
    own, lib, n = res["ex_m1"]
    assert n > 1_000_000 and own <= 2.0, (own, lib)
    own, lib, n = res["sqrt_nr"]
    assert own <= 1.0, (own, lib)
    bad, _, n = res["split_df"]
    assert n > 3_000_000 and bad == 0, bad
    bad, _, n = res["f32_f64_of"]
    assert n > 2_000_000 and bad == 0, bad

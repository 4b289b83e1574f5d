"""The mixed-precision push converts between binary64 and binary32 with
integer operations (the double-precision unit is narrow on this GPU).  This
builds a small CUDA program that checks those conversions bit for bit against
the conversion instructions: all 2^32 floats to double, and 2^30 doubles
(random patterns, the float exponent range, exact rounding ties and their
neighbours, zone-centre offsets) to float and through the NaN test."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_integer_pipe_conversions_match_conversion_instructions():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(ROOT, "tests", "cuda", "conversions_check.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "conv")
        subprocess.check_call([nvcc, "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-I", os.path.join(ROOT, "include"),
                               "-I", os.path.join(ROOT, "paper_1908_10793_gb300", "csrc"),
                               "-o", exe, src])
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "f32_to_f64 mismatches 0" in r.stdout and "f64_to_f32 mismatches 0" in r.stdout

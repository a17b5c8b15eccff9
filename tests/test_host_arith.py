"""Host checks of device helpers that are written to be host-callable (no GPU).

f2d_exact (arith.cuh) converts float to double with integer operations only, so
the double-float kernels' results never touch GB300's FP64 pipe; it must equal
the hardware conversion on every float, including zeros, subnormals, infinities
and NaNs.  df2d_exact turns a double-float pair into the double nearest to its
exact sum the same way (FP32 adds and integer operations), and must equal the
IEEE double sum of the two converted floats bit for bit.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_06971_gb300", "csrc")


@pytest.mark.timeout(600)
def test_f2d_exact_all_floats(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "f2d_exact_check")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(ROOT, "tests", "f2d_exact_check.cu")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=560)
    assert r.returncode == 0 and "mismatches: 0" in r.stdout, r.stdout


@pytest.mark.timeout(600)
def test_df2d_exact_matches_fp64_sum(tmp_path):
    """df2d_exact (arith.cuh) turns a double-float (hi, lo) into the double nearest to hi + lo with
    FP32 adds and integer operations; it must equal the IEEE double sum bit for bit, ties included."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "df2d_exact_check")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(ROOT, "tests", "df2d_exact_check.cu")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=560)
    assert r.returncode == 0 and "mismatches: 0" in r.stdout, r.stdout

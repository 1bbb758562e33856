"""The mixed path's float-float arithmetic, checked on the host against exact references.
- The integer conversion of a float-float pair to FP64, used by the augmented kernel for its
  FP64 result and moments, must give the bits of the FP64 addition hi + lo (round to nearest
  even). Checked on random pairs over a wide range of exponent gaps and on the borrow, carry,
  tie and special cases.
- TwoSum and TwoProduct must be exact.
- The float-float add, fast add and multiply, and the stencil neighbour sum must stay within
  their error bounds, measured against quad-precision sums of the float parts.
The helpers are host/device inline functions, so the check compiles them as host code."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1611_05677_gb300", "csrc")


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return path if os.path.exists(path) else None


def test_float_float_helpers(tmp_path):
    cc = nvcc()
    if cc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "ff_conversion_check")
    src = os.path.join(ROOT, "tests", "ff_conversion_check.cu")
    subprocess.run([cc, "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", exe, src],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe, "500000"], capture_output=True, text=True, timeout=300)
    checked, bad = (int(v) for v in out.stdout.split()[-2:])
    assert checked >= 2_000_000
    assert bad == 0, out.stdout
    assert out.returncode == 0

"""Host check of the double-float arithmetic used by the OSB_DF64 path
(tests/dd_check.cu against long double): conversion from double within
2^-49 relative with the head equal to the double rounded to FP32, the sum
within 3u^2, the product within 5u^2 and the quotient within 16u^2
(u = 2^-24, Joldes-Muller-Popescu bounds), the stencil accumulator within
16u^2 of the operands' magnitude."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_arithmetic_error_bounds(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "dd_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off", "-o", exe,
                    os.path.join(ROOT, "tests", "dd_check.cu"),
                    "-I", os.path.join(ROOT, "paper_1609_01277_gb300", "csrc")],
                   check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout

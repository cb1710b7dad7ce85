"""The FP32 path converts float <-> double with integer instructions
(f2d_bits, d2f_bits).  Pin them to the compiler's IEEE conversions on the
host: every float widened exactly, 16 M doubles over all exponents narrowed
round-to-nearest-even (ties and carries included), with the documented flush
of sub-normal results to signed zero; NaNs stay NaNs of the same sign."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_pipe_conversions_match_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "conv_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "conv_check.cu"),
                    "-I", os.path.join(ROOT, "paper_1609_01277_gb300", "csrc"), "-I", os.path.join(ROOT, "include")],
                   check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    assert "0 mismatches" in r.stdout

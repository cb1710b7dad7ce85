"""The C ABI from a plain C11 program (tests/c_abi_tgv.c): it compiles and
links against include/osb.h and libosb.so with gcc (no GPU needed), and on a
GPU it runs a 24^3 Taylor-Green case whose kinetic energy matches the oracle."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_tgv.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(tmp_path):
    from paper_1609_01277_gb300 import build
    lib = build.build()
    if not shutil.which("gcc") or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime_api.h")):
        pytest.skip("gcc or the CUDA runtime headers missing")
    exe = str(tmp_path / "c_abi_tgv")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I",
           os.path.join(CUDA, "include"), SRC, "-o", exe, "-L", libdir, "-losb", "-L", os.path.join(CUDA, "lib64"),
           "-lcudart", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_compiles_and_links(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_program_runs(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr)
    vals = dict(kv.split("=") for kv in r.stdout.split())
    from oracle import oracle as orc
    case = orc.Case(24, 24, 24, order=4)
    Q = orc.tgv_init(case)
    ke0 = orc.diagnostics(case, Q)["ke"]
    ke10 = orc.diagnostics(case, orc.rk3_step(case, Q, 10))["ke"]
    assert int(vals["steps"]) == 10
    assert abs(float(vals["series0"]) - ke0) < 1e-13 * ke0
    assert abs(float(vals["ke"]) - ke10) < 1e-12 * ke10

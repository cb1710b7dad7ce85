"""Builds libosb.so in-tree with nvcc for sm_103a (GB300).

One translation unit per stencil order plus the misc kernels and the C ABI,
compiled in parallel, then linked into ``paper_1609_01277_gb300/_lib/libosb.so``.
``-Xptxas -v`` output (registers, spills, shared memory) goes to
``_lib/ptxas.log``.

``build(bounds_check=True)`` builds the same sources with -DOSB_BOUNDS_CHECK
into ``_lib_bc/libosb.so``: every index a stage kernel forms is tested against
its buffer, a failure is recorded in the grid's device error word
(osb_diagnostics then returns OSB_ERR_BOUNDS) and the access is kept inside
the buffer.  A test build, slower than the product build.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libosb.so")
OUT_BC = os.path.join(HERE, "_lib_bc")
LIB_BC = os.path.join(OUT_BC, "libosb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-Xptxas", "-v",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "osb.h")]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, jobs: int | None = None, bounds_check: bool = False) -> str:
    out, lib = (OUT_BC, LIB_BC) if bounds_check else (OUT, LIB)
    flags = FLAGS + (["-DOSB_BOUNDS_CHECK"] if bounds_check else [])
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    srcs = _sources()
    objs = [os.path.join(out, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def compile_one(pair):
        src, obj = pair
        r = subprocess.run([cc, *ARCH, *flags, "-c", src, "-o", obj], capture_output=True, text=True)
        return src, r

    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 4)) as ex:
        for src, r in ex.map(compile_one, zip(srcs, objs)):
            logs.append(f"== {os.path.basename(src)}\n{r.stdout}{r.stderr}")
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    with open(os.path.join(out, "ptxas.log"), "w") as f:
        f.write("\n".join(logs))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))

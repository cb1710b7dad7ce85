"""The C-ABI library loads, exports every entry point include/osb.h declares,
and rejects bad arguments before touching the GPU (no compute calls here)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def osb():
    from paper_1609_01277_gb300 import build
    build.build()
    from paper_1609_01277_gb300 import osb as m
    m.load()
    return m


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(osb_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(osb):
    L = osb.load()
    declared = _declared()
    assert "osb_rk3_step" in declared and "osb_grid_create" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert set(osb.EXPORTS) <= declared


def test_status_strings(osb):
    L = osb.load()
    for code in range(8):
        assert L.osb_status_string(code)
    assert L.osb_status_string(0) == b"ok"


def _create(osb, desc, params, sptr=256, sb=None, wptr=512, wb=None):
    L = osb.load()
    sb = L.osb_state_bytes(ctypes.byref(desc)) if sb is None else sb
    wb = L.osb_workspace_bytes(ctypes.byref(desc)) if wb is None else wb
    h = ctypes.c_void_p()
    st = L.osb_grid_create(ctypes.byref(desc), ctypes.byref(params), sptr, sb, wptr, wb, None, ctypes.byref(h))
    return st, h


def test_sizes(osb):
    L = osb.load()
    d = osb.GridDesc(32, 32, 32, 4, osb.OSB_FP64, 0)
    n = 32 ** 3
    assert L.osb_state_bytes(ctypes.byref(d)) == 20 * n * 8
    d32 = osb.GridDesc(32, 32, 32, 4, osb.OSB_FP32, 0)
    assert L.osb_state_bytes(ctypes.byref(d32)) == 10 * n * 8 + 10 * n * 4
    ddd = osb.GridDesc(32, 32, 32, 4, osb.OSB_DF64, 0)   # double-float registers: 8 bytes per value
    assert L.osb_state_bytes(ctypes.byref(ddd)) == 20 * n * 8
    assert L.osb_workspace_bytes(ctypes.byref(d)) > 15 * n * 8
    bad = osb.GridDesc(32, 32, 32, 5, osb.OSB_FP64, 0)
    assert L.osb_state_bytes(ctypes.byref(bad)) == 0
    assert L.osb_workspace_bytes(ctypes.byref(bad)) == 0


def test_point_count_bound(osb):
    """Grids hold at most 2^31 - 1 points (the point count is a 32-bit int in
    the kernels' index arithmetic; their grid-stride loops run in 64 bits, so
    the last stride past n cannot wrap): 1 x 1 x (2^31 - 1) is sized, one
    point more is refused by every size query."""
    L = osb.load()
    top = (1 << 31) - 1
    ok = osb.GridDesc(1, 1, top, 2, osb.OSB_FP64, 0)
    sb = L.osb_state_bytes(ctypes.byref(ok))
    assert sb >= 20 * top * 8 and sb - 20 * top * 8 < 20 * 256
    assert L.osb_workspace_bytes(ctypes.byref(ok)) > 0
    for dims in ((1, 1, 1 << 31), (2, 1 << 15, 1 << 15), (46341, 46341, 1)):
        over = osb.GridDesc(*dims, 2, osb.OSB_FP64, 0)
        assert dims[0] * dims[1] * dims[2] > top
        assert L.osb_state_bytes(ctypes.byref(over)) == 0
        assert L.osb_workspace_bytes(ctypes.byref(over)) == 0


@pytest.mark.parametrize("desc", [
    (0, 8, 8, 4, 0, 0), (8, 8, 8, 3, 0, 0), (8, 8, 8, 14, 0, 0), (8, 8, 8, 0, 0, 0),
    (8, 8, 8, 4, 3, 0), (8, 8, 8, 4, 0, 7), (2048, 2048, 1024, 4, 0, 0)])
def test_invalid_descriptor_rejected(osb, desc):
    st, h = _create(osb, osb.GridDesc(*desc), osb.Params(1600, 0.1, 1.4, 0.71, 1e-3), sb=1 << 40, wb=1 << 40)
    assert st == 1 and not h.value


@pytest.mark.parametrize("params", [(0, 0.1, 1.4, 0.71, 1e-3), (1600, -0.1, 1.4, 0.71, 1e-3),
                                    (1600, 0.1, 1.0, 0.71, 1e-3), (1600, 0.1, 1.4, 0.0, 1e-3),
                                    (1600, 0.1, 1.4, 0.71, 0.0), (float("nan"), 0.1, 1.4, 0.71, 1e-3)])
def test_invalid_params_rejected(osb, params):
    st, _ = _create(osb, osb.GridDesc(8, 8, 8, 4, 0, 0), osb.Params(*params))
    assert st == 1


def test_buffer_checks(osb):
    d = osb.GridDesc(8, 8, 8, 4, 0, 0)
    p = osb.Params(1600, 0.1, 1.4, 0.71, 1e-3)
    st, _ = _create(osb, d, p, sptr=256 + 8)           # misaligned
    assert st == 6
    st, _ = _create(osb, d, p, sb=100)                 # too small
    assert st == 6
    st, _ = _create(osb, d, p, wb=100)
    assert st == 6
    st, _ = _create(osb, d, p, sptr=0)                 # NULL
    assert st == 1
    L = osb.load()
    assert L.osb_rk3_step(None, 1) == 1
    assert L.osb_diagnostics(None, None) == 1
    assert L.osb_batch_step(None, 1, 1) == 1
    assert L.osb_set_boundaries(None, 0, 0, 0) == 1
    assert L.osb_set_diag_series(None, None, 0) == 1
    assert L.osb_diag_series_count(None, None) == 1


def test_binding_refuses_missing_library(osb, tmp_path):
    import importlib
    m = importlib.import_module("paper_1609_01277_gb300.osb")
    saved = m._lib
    try:
        m._lib = None
        with pytest.raises(RuntimeError):
            m.load(str(tmp_path / "missing.so"))
    finally:
        m._lib = saved


def test_noalloc_diagnostics_rejects_bad_arguments_before_gpu_work(osb):
    """Argument checks of the allocation-free diagnostics run on the host,
    before any CUDA call (fake, aligned, never-dereferenced pointers)."""
    L = osb.load()
    p = osb.Params(1600, 0.1, 1.4, 0.71, 1e-3)
    ok_ptr = 4096
    assert L.osb_diagnostics_noalloc(None, 8, 8, 8, 4, ctypes.byref(p), ok_ptr, None) == 1
    assert L.osb_diagnostics_noalloc(ok_ptr, 8, 8, 8, 4, ctypes.byref(p), ok_ptr + 4, None) == 6
    assert L.osb_diagnostics_noalloc(ok_ptr, 0, 8, 8, 4, ctypes.byref(p), ok_ptr, None) == 1
    assert L.osb_diagnostics_noalloc(ok_ptr, 8, 8, 8, 5, ctypes.byref(p), ok_ptr, None) == 1
    assert L.osb_diagnostics_noalloc(ok_ptr, 2048, 2048, 1024, 4, ctypes.byref(p), ok_ptr, None) == 1
    assert b"too large" in L.osb_last_error()
    bad = osb.Params(1600, 0.1, 1.0, 0.71, 1e-3)
    assert L.osb_diagnostics_noalloc(ok_ptr, 8, 8, 8, 4, ctypes.byref(bad), ok_ptr, None) == 1


def test_scalar_rejects_bad_arguments_before_gpu_work(osb):
    L = osb.load()
    a = (ctypes.c_double * 3)(1.0, 0.0, 0.0)
    ok = 4096  # never dereferenced: every call below fails its argument checks
    assert L.osb_scalar_rk3(None, ok, None, 8, 8, 8, 4, a, 0.1, 1e-3, 1, None) == 1
    assert L.osb_scalar_rk3(ok, ok, None, 0, 8, 8, 4, a, 0.1, 1e-3, 1, None) == 1
    assert L.osb_scalar_rk3(ok, ok, None, 8, 8, 8, 3, a, 0.1, 1e-3, 1, None) == 1
    assert L.osb_scalar_rk3(ok, ok, None, 8, 8, 8, 14, a, 0.1, 1e-3, 1, None) == 1
    assert L.osb_scalar_rk3(ok, ok, None, 8, 8, 8, 4, a, -0.1, 1e-3, 1, None) == 1
    assert L.osb_scalar_rk3(ok, ok, None, 8, 8, 8, 4, a, 0.1, 0.0, 1, None) == 1
    assert L.osb_scalar_rk3(ok, ok, None, 8, 8, 8, 4, a, 0.1, 1e-3, -1, None) == 1
    assert L.osb_scalar_rk3(ok + 4, ok, None, 8, 8, 8, 4, a, 0.1, 1e-3, 1, None) == 6
    assert L.osb_scalar_rk3(ok, ok, None, 8, 8, 8, 4, a, 0.1, 1e-3, 0, None) == 0  # nothing to do



def test_batch_autotune_and_tile_depth_reject_bad_arguments_before_gpu_work(osb):
    L = osb.load()
    assert L.osb_autotune_batch(None, 1, 2) == 1
    assert L.osb_tile_depth(None) == 0
    bad = osb.GridDesc(8, 8, 8, 5, osb.OSB_FP64, 0)
    assert L.osb_tile_depth(ctypes.byref(bad)) == 0
    d32 = osb.GridDesc(40, 40, 40, 4, osb.OSB_FP32, 0)
    d64 = osb.GridDesc(40, 40, 40, 4, osb.OSB_FP64, 0)
    assert L.osb_tile_depth(ctypes.byref(d32)) >= 1 and L.osb_tile_depth(ctypes.byref(d64)) >= 1


def test_z_slab_calls_reject_null_grids(osb):
    L = osb.load()
    assert L.osb_set_z_slab(None, 64) == 1
    assert L.osb_halo_bytes(None) == 0
    assert L.osb_halo_pack(None, 0, 256, 512) == 1
    assert L.osb_halo_unpack(None, 0, 256, 512) == 1
    assert L.osb_rk3_stage(None, 0) == 1

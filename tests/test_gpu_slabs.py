"""z-slab decomposition inside the library, on one GPU.

A periodic box of nz planes is split into W slabs (z-slab grids with `order`
ghost planes at each end, osb_set_z_slab); before every RK stage each slab
packs the planes next to its faces (osb_halo_pack, the halo pack kernel),
the staging buffers go to the z neighbours (here device copies on the same
stream; across GPUs NCCL send/recv), each slab unpacks what it received into
its ghost planes (osb_halo_unpack) and runs the stage (osb_rk3_stage).  The
owned planes must evolve exactly as in the undivided box: same operands, same
order of operations, so the same bits, in every precision and stage form.
The per-slab diagnostics over the owned planes, weighted by the slab sizes,
must give the diagnostics of the whole box (one all-reduce in the multi-GPU
design).
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1609_01277_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01277_gb300 import build
    build.build()
    from paper_1609_01277_gb300 import osb as m
    m.load()
    return m


def _slabs(osb, Q, dims, W, order, prec, **kw):
    nx, ny, nz = dims
    H, nown = order, nz // W
    grids = []
    for w in range(W):
        g = osb.Grid(osb.Config(nx, ny, nown + 2 * H, order=order, precision=prec, **kw))
        g.set_z_slab(nz)
        planes = [(w * nown - H + k) % nz for k in range(nown + 2 * H)]
        g.set_state(np.ascontiguousarray(Q[:, planes]))
        grids.append(g)
    return grids


def _exchange(torch, grids, source, bufs):
    W = len(grids)
    send, recv = bufs
    for g, (lo, hi) in zip(grids, send):
        g.halo_pack(source, lo, hi)
    for s in range(W):
        recv[s][0].copy_(send[(s - 1) % W][1])   # below: the low neighbour's high face
        recv[s][1].copy_(send[(s + 1) % W][0])   # above: the high neighbour's low face
    for g, (lo, hi) in zip(grids, recv):
        g.halo_unpack(source, lo, hi)


def _buffers(torch, grids):
    nb = grids[0].halo_bytes()
    mk = lambda: torch.empty(nb // 8, dtype=torch.float64, device="cuda")
    return [(mk(), mk()) for _ in grids], [(mk(), mk()) for _ in grids]


def _run(torch, grids, steps):
    bufs = _buffers(torch, grids)
    for _ in range(steps):
        for k in range(3):
            _exchange(torch, grids, k, bufs)
            for g in grids:
                g.stage(k)
    return bufs


def _owned(grids, order):
    H = order
    return np.concatenate([g.get_state()[:, H:-H] for g in grids], axis=1)


@pytest.mark.parametrize("W", [2, 4])
@pytest.mark.parametrize("prec_name,order", [("fp64", 4), ("fp64", 2), ("fp32", 4), ("fp32", 8), ("df64", 4)])
def test_slabs_reproduce_the_whole_box_bitwise(osb, W, prec_name, order):
    import torch
    prec = {"fp64": osb.OSB_FP64, "fp32": osb.OSB_FP32, "df64": osb.OSB_DF64}[prec_name]
    dims = (24, 20, 32) if order <= 4 else (40, 16, 48)
    nx, ny, nz = dims
    kw = dict(Re=400.0, Mach=0.2, dt=1.5e-3)
    full = osb.Grid(osb.Config(nx, ny, nz, order=order, precision=prec, **kw))
    full.init_taylor_green(inputs.gaussian_noise(nx, ny, nz, seed=17), 1e-2)
    Q0 = full.get_state()
    full.step(3)
    grids = _slabs(osb, Q0, dims, W, order, prec, **kw)
    _run(torch, grids, 3)
    assert np.array_equal(_owned(grids, order), full.get_state())
    assert grids[0].diagnostics()["step"] == 3


def test_slab_diagnostics_combine_to_the_whole_box(osb):
    import torch
    dims, order, W = (24, 20, 32), 4, 4
    nx, ny, nz = dims
    full = osb.Grid(osb.Config(nx, ny, nz, order=order, Re=400.0, dt=1.5e-3))
    full.init_taylor_green(inputs.gaussian_noise(nx, ny, nz, seed=23), 1e-2)
    grids = _slabs(osb, full.get_state(), dims, W, order, osb.OSB_FP64, Re=400.0, dt=1.5e-3)
    full.step(2)
    bufs = _run(torch, grids, 2)
    _exchange(torch, grids, 3, bufs)     # ghost planes of the accumulator for the enstrophy stencils
    ref = full.diagnostics()
    parts = [g.diagnostics() for g in grids]
    for key in ("ke", "enstrophy"):
        got = sum(p[key] for p in parts) / W
        assert got == pytest.approx(ref[key], rel=1e-13)
    for m in range(5):
        got = sum(p["total"][m] for p in parts) / W
        assert got == pytest.approx(ref["total"][m], rel=1e-13, abs=1e-15)
    assert max(p["max_cfl"] for p in parts) == pytest.approx(ref["max_cfl"], rel=1e-14)


def test_slab_ghosts_left_stale_change_the_owned_planes(osb):
    """Skipping the exchange before one stage leaves ghost planes of the
    previous stage's source: the owned planes next to the faces go wrong, so
    the bitwise test above depends on every exchange."""
    import torch
    dims, order, W = (24, 20, 32), 4, 2
    nx, ny, nz = dims
    full = osb.Grid(osb.Config(nx, ny, nz, order=order, Re=400.0, dt=1.5e-3))
    full.init_taylor_green(inputs.gaussian_noise(nx, ny, nz, seed=29), 1e-2)
    grids = _slabs(osb, full.get_state(), dims, W, order, osb.OSB_FP64, Re=400.0, dt=1.5e-3)
    full.step(1)
    bufs = _buffers(torch, grids)
    for k in range(3):
        if k != 1:
            _exchange(torch, grids, k, bufs)
        for g in grids:
            g.stage(k)
    got = _owned(grids, order)
    ref = full.get_state()
    assert not np.array_equal(got[:, :order], ref[:, :order])            # next to a face
    mid = slice(2 * order, nz // W - 2 * order)
    assert np.array_equal(got[:, mid], ref[:, mid])                       # far from the faces


def test_slab_calls_reject_bad_arguments(osb):
    import torch
    L = osb.load()
    g = osb.Grid(osb.Config(16, 16, 24, order=4))
    h = g.handle
    buf = torch.empty(1 << 16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert L.osb_halo_bytes(h) == 0                      # not a slab yet
    assert L.osb_halo_pack(h, 0, p, p + 8192) == 1       # not a slab
    assert L.osb_set_z_slab(h, 0) == 1                   # nz_domain >= 1
    assert L.osb_set_z_slab(h, 64) == 0
    assert L.osb_halo_bytes(h) == 5 * 4 * 16 * 16 * 8
    assert L.osb_halo_pack(h, 4, p, p + 8192) == 1       # source 0..3
    assert L.osb_halo_pack(h, 1, p, p + 8192) == 1       # stage 1's source before stage 0 ran
    assert L.osb_halo_pack(h, 3, p + 4, p + 8192) == 6   # unaligned buffer
    assert L.osb_halo_pack(h, 3, None, p) == 1
    assert L.osb_rk3_stage(h, 2) == 1                    # stages in order
    assert L.osb_rk3_step(h, 1) == 2                     # slabs step one stage at a time
    assert L.osb_euler_step(h, 1) == 2
    assert L.osb_set_boundaries(h, 0, 0, 1) == 2
    small = osb.Grid(osb.Config(16, 16, 11, order=4))
    assert L.osb_set_z_slab(small.handle, 64) == 1      # nz < 3 * order

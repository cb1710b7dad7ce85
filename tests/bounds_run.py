"""Runs every stage path of the bounds-check build of libosb (-DOSB_BOUNDS_CHECK)
on small, ragged and degenerate grids and prints one JSON object: the status
osb_diagnostics returned after each case (0 = no index fell outside its
buffer), and the FP64 state of one case for a parity check.  Run in its own
process (python -m tests.bounds_run) so that it loads the check build."""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main() -> int:
    import torch
    from paper_1609_01277_gb300 import build, inputs
    lib = build.build(bounds_check=True)
    from paper_1609_01277_gb300 import osb
    osb.load(lib)
    out = {}

    def status(g):
        d = osb.Diag()
        return int(osb.load().osb_diagnostics(g.handle, ctypes.byref(d)))

    import ctypes

    def run(name, nx, ny, nz, order, prec=osb.OSB_FP64, steps=2, env=None, bc=None, visc=0, euler=False):
        saved = {k: os.environ.get(k) for k in (env or {})}
        os.environ.update(env or {})
        try:
            kw = dict(order=order, precision=prec, Re=300.0, dt=1e-3, visc_form=visc)
            if bc:
                kw["bc"] = bc
            g = osb.Grid(osb.Config(nx, ny, nz, **kw))
            g.init_taylor_green(inputs.gaussian_noise(nx, ny, nz, seed=nx + ny + nz), 1e-3)
            if euler:
                g.euler_step(steps)
            else:
                g.step(steps)
            g.residual()
            out[name] = status(g)
            return g
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    F64, F32, D64 = osb.OSB_FP64, osb.OSB_FP32, osb.OSB_DF64
    for order in (2, 4, 6, 8, 10, 12):
        run(f"fp64_o{order}_9x7x5", 9, 7, 5, order)
    for dims in ((1, 1, 1), (5, 1, 1), (1, 7, 1), (1, 1, 6), (3, 4, 2)):
        run(f"fp64_o8_{dims}", *dims, 8)
        run(f"fp32_o2_{dims}", *dims, 2, F32)
        run(f"fp32_o4_{dims}", *dims, 4, F32)
        run(f"df64_o4_{dims}", *dims, 4, D64)
    for dims, order in (((37, 20, 9), 2), ((72, 24, 16), 4), ((70, 9, 33), 4), ((96, 40, 20), 2),
                        ((40, 24, 20), 6), ((104, 32, 20), 8), ((36, 12, 10), 8)):
        run(f"fp32_o{order}_{dims}", *dims, order, F32)
        run(f"fp32_o{order}_{dims}_cpasync", *dims, order, F32, env={"OSB_FP32_LOADS": "cpasync"})
    run("fp32_o10_split3", 24, 16, 12, 10, F32, env={"OSB_FP32_STAGE": "split3"})
    run("fp32_o4_zmarch", 72, 24, 16, 4, F32, env={"OSB_FP32_STAGE": "zmarch"})
    run("fp32_o8_wide_residual", 104, 32, 20, 8, F32, env={"OSB_FP32_ZRHS": "wide"})
    run("fp64_o4_formB", 20, 12, 10, 4, visc=1)
    run("fp64_o4_euler", 20, 12, 10, 4, euler=True)
    run("fp32_o4_euler", 72, 24, 16, 4, F32, euler=True)
    S = (osb.OSB_BC_SYMMETRIC,) * 3
    run("fp64_o4_octant", 8, 8, 8, 4, bc=S)
    run("fp32_o6_octant", 8, 6, 5, 6, F32, bc=S)
    # z slabs: 2 slabs of a 24 x 20 x 32 box, FP64 and FP32 (fused)
    for prec, tag in ((F64, "fp64"), (F32, "fp32")):
        H, W, nz = 4, 2, 32
        grids = []
        full = osb.Grid(osb.Config(24, 20, nz, order=4, precision=prec))
        full.init_taylor_green(inputs.gaussian_noise(24, 20, nz, seed=3), 1e-3)
        Q = full.get_state()
        for w in range(W):
            g = osb.Grid(osb.Config(24, 20, nz // W + 2 * H, order=4, precision=prec))
            g.set_z_slab(nz)
            g.set_state(np.ascontiguousarray(Q[:, [(w * nz // W - H + k) % nz for k in range(nz // W + 2 * H)]]))
            grids.append(g)
        nb = grids[0].halo_bytes() // 8
        bufs = [[torch.empty(nb, dtype=torch.float64, device="cuda") for _ in range(4)] for _ in grids]
        for k in range(3):
            for g, b in zip(grids, bufs):
                g.halo_pack(k, b[0], b[1])
            for s in range(W):
                bufs[s][2].copy_(bufs[(s - 1) % W][1])
                bufs[s][3].copy_(bufs[(s + 1) % W][0])
            for g, b in zip(grids, bufs):
                g.halo_unpack(k, b[2], b[3])
            for g in grids:
                g.stage(k)
        for w, g in enumerate(grids):
            out[f"slab_{tag}_{w}"] = status(g)
    # ensembles: three-kernel items (FP64) and z-march items (FP32) of the
    # persistent kernel, FP32 step graphs on concurrent streams
    for prec, tag, mode in ((F64, "fp64", "persistent"), (F32, "fp32", "persistent"), (F32, "fp32s", "streams")):
        os.environ["OSB_BATCH_MODE"] = mode
        ens = []
        for i, n in enumerate((12, 20, 16)):
            g = osb.Grid(osb.Config(n, n, n, order=4, precision=prec, dt=1e-3))
            g.init_taylor_green(inputs.gaussian_noise(n, n, n, seed=i), 1e-3)
            ens.append(g)
        osb.batch_step(ens, 2)
        for i, g in enumerate(ens):
            out[f"batch_{tag}_{i}"] = status(g)
    os.environ.pop("OSB_BATCH_MODE", None)
    g = run("parity_fp64_o4_13x11x9", 13, 11, 9, 4, steps=3)
    out["_state"] = g.get_state().tolist()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())

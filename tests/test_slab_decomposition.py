"""Domain decomposition of the time step into z-slabs, one rank per slab, on
CPU ranks over torch.distributed (gloo, world size 2 and 4).

Each rank owns nz/W planes.  Before every RK stage it exchanges 2R ghost
planes of the stage source with its z-neighbours (R from the first-derivative
stencils, doubled by the nested viscous-work and D_i(div u) terms of form A),
evaluates the residual on its slab plus ghosts and applies the low-storage
update (Section 2.4 time stepping, Section 3.3 equations) to its own planes.
The residual of an owned plane reads data at most 2R planes away, so the
slab's own planes must reproduce the single-domain oracle bit for bit; the
kinetic energy and conserved totals are reduced across ranks with one
all-reduce per step and agree with the single-domain sums to rounding.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs

N, ORDER, STEPS = 16, 4, 3
PARAMS = dict(Re=800.0, Mach=0.2, dt=2e-3)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange(q: np.ndarray, H: int) -> np.ndarray:
    """Slab with H ghost planes on each side from the periodic z-neighbours:
    each rank sends its first H planes to the rank below and its last H planes
    to the rank above, and receives the matching faces (neighbour send/recv,
    as NCCL would carry them between GPUs)."""
    import torch
    rank, world = dist.get_rank(), dist.get_world_size()
    below_rank, above_rank = (rank - 1) % world, (rank + 1) % world
    lo = torch.from_numpy(np.ascontiguousarray(q[:, :H]))
    hi = torch.from_numpy(np.ascontiguousarray(q[:, -H:]))
    below, above = torch.empty_like(hi), torch.empty_like(lo)
    reqs = [dist.isend(lo, below_rank, tag=1), dist.isend(hi, above_rank, tag=2),
            dist.irecv(below, below_rank, tag=2), dist.irecv(above, above_rank, tag=1)]
    for r in reqs:
        r.wait()
    return np.ascontiguousarray(np.concatenate([below.numpy(), q, above.numpy()], axis=1))


def _worker(rank: int, world: int, port: int, out_dir: str):
    import torch
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        orc.set_threads(1)
        full = orc.Case(N, N, N, order=ORDER, **PARAMS)
        Q0 = orc.tgv_init(full, inputs.gaussian_noise(N, N, N, 5), 1e-3)
        nzl = N // world
        H = ORDER  # 2R ghost planes
        slab = orc.Case(N, N, nzl + 2 * H, order=ORDER, nz_domain=N, **PARAMS)
        alpha, beta = orc.rk3_coeffs()
        y = np.ascontiguousarray(Q0[:, rank * nzl:(rank + 1) * nzl])
        ke_series = []
        for _ in range(STEPS):
            q = y.copy()
            for k in range(3):
                R = orc.residual(slab, _exchange(q, H))[:, H:H + nzl]
                a, b = alpha[k] * full.dt, beta[k] * full.dt
                q = y + a * R
                y = y + b * R
            # per-step reduction of E_k and the conserved totals (one all-reduce)
            rho = y[0]
            part = np.array([0.5 * np.sum((y[1] ** 2 + y[2] ** 2 + y[3] ** 2) / rho)] +
                            [np.sum(y[m]) for m in range(5)])
            t = torch.from_numpy(part)
            dist.all_reduce(t)
            ke_series.append(t.numpy() / N ** 3)
        np.save(os.path.join(out_dir, f"slab{rank}.npy"), y)
        if rank == 0:
            np.save(os.path.join(out_dir, "reduced.npy"), np.array(ke_series))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_z_slab_halo_exchange_matches_single_domain(tmp_path, world):
    orc.build()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    full = orc.Case(N, N, N, order=ORDER, **PARAMS)
    Q = orc.tgv_init(full, inputs.gaussian_noise(N, N, N, 5), 1e-3)
    series = []
    for _ in range(STEPS):
        Q = orc.rk3_step(full, Q, 1)
        d = orc.diagnostics(full, Q)
        series.append([d["ke"]] + [float(np.mean(Q[m])) for m in range(5)])
    slabs = np.concatenate([np.load(tmp_path / f"slab{r}.npy") for r in range(world)], axis=1)
    assert np.array_equal(slabs, Q)          # bit for bit
    red = np.load(tmp_path / "reduced.npy")
    ref = np.array(series)
    assert np.allclose(red, ref, rtol=1e-13, atol=1e-15)


def test_slab_needs_both_ghost_widths():
    """With only R ghost planes (no room for the nested terms) the owned planes
    next to the slab faces go wrong: the 2R width is necessary, not slack."""
    orc.build()
    full = orc.Case(N, N, N, order=ORDER, **PARAMS)
    Q0 = orc.tgv_init(full, inputs.gaussian_noise(N, N, N, 5), 1e-3)
    ref = orc.residual(full, Q0)
    nzl, H = N // 2, ORDER // 2
    ext = np.concatenate([Q0[:, -H:], Q0[:, :nzl], Q0[:, nzl:nzl + H]], axis=1)
    slab = orc.Case(N, N, nzl + 2 * H, order=ORDER, nz_domain=N, **PARAMS)
    R = orc.residual(slab, np.ascontiguousarray(ext))[:, H:H + nzl]
    assert not np.array_equal(R[:, :1], ref[:, :1])        # face plane depends on planes 2R away
    assert np.array_equal(R[:, H:nzl - H], ref[:, H:nzl - H])  # interior planes are unaffected

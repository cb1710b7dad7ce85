"""Per-step diagnostics series fused into the first RK stage (osb_set_diag_series).

Each entry is the kinetic energy and enstrophy (Section 3.3 grid means) of
the state at the start of a step.  They are compared with the separate
diagnostics reduction (osb_diagnostics) on the same states and with the CPU
oracle: FP64 and double-float to rounding, FP32 within its FP32 bound.  Also:
CUDA-graph replays (multi-step calls), forward Euler steps, the ring's
wrap-around, symmetric grids, detaching, and the ensemble's refusal.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as orc
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


def _reference_series(osb, cfg, noise, steps, euler=False):
    """ke, enstrophy of the states Q^0 .. Q^{steps-1} from osb_diagnostics on
    a second grid stepped one step at a time (FP64 accumulator)."""
    g = osb.Grid(cfg)
    g.init_taylor_green(noise, 1e-2 if noise is not None else 0.0)
    out = []
    for _ in range(steps):
        d = g.diagnostics()
        out.append((d["ke"], d["enstrophy"]))
        g.euler_step(1) if euler else g.step(1)
    return np.array(out)


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (2, 1e-12), (1, 2e-6)])
@pytest.mark.parametrize("order", [4, 8])
def test_series_matches_diagnostics(osb, precision, tol, order):
    import torch
    n, steps = 24, 6
    noise = torch.from_numpy(inputs.gaussian_noise(n, n, n, 5)).cuda()
    cfg = osb.Config(n, n, n, order=order, precision=precision, Re=400.0)
    g = osb.Grid(cfg)
    g.init_taylor_green(noise, 1e-2)
    g.set_diag_series(16)
    g.step(1)            # direct launches
    g.step(steps - 1)    # captured step graph
    s = g.diag_series()
    assert s.shape == (steps, 2)
    ref = _reference_series(osb, cfg, noise, steps)
    assert np.max(np.abs(s - ref) / np.abs(ref)) < tol, (s, ref)


def test_series_matches_oracle_and_euler(osb):
    n = 16
    cfg = osb.Config(n, n, n, order=4, Re=200.0, dt=2e-3)
    g = osb.Grid(cfg)
    g.init_taylor_green()
    g.set_diag_series(8)
    g.euler_step(3)
    s = g.diag_series()
    case = orc.Case(n, n, n, order=4, Re=200.0, dt=2e-3)
    Q = orc.tgv_init(case)
    for k in range(3):
        d = orc.diagnostics(case, Q)
        assert abs(s[k, 0] - d["ke"]) <= 1e-13 * d["ke"]
        assert abs(s[k, 1] - d["enstrophy"]) <= 1e-12 * d["enstrophy"]
        Q = orc.euler_step(case, Q, 1)


def test_ring_wraps_and_detaches(osb):
    n = 16
    cfg = osb.Config(n, n, n, order=4)
    g = osb.Grid(cfg)
    g.init_taylor_green()
    g.set_diag_series(3)
    g.step(7)
    s = g.diag_series()
    ref = _reference_series(osb, cfg, None, 7)
    assert s.shape == (3, 2)
    assert np.max(np.abs(s - ref[4:]) / ref[4:]) < 1e-13
    g.set_diag_series(None)
    g.step(2)  # no recording, no fault
    g.set_diag_series(4)
    g.step(1)
    assert g.diag_series().shape == (1, 2)


def test_symmetric_grid_series(osb):
    n = 12
    sym = (osb.OSB_BC_SYMMETRIC,) * 3
    cfg = osb.Config(n, n, n, order=4, bc=sym)
    g = osb.Grid(cfg)
    g.init_taylor_green()
    g.set_diag_series(4)
    g.step(3)
    ref = _reference_series(osb, cfg, None, 3)
    assert np.max(np.abs(g.diag_series() - ref) / ref) < 1e-13


def test_batch_refuses_series_grids(osb):
    n = 16
    g = osb.Grid(osb.Config(n, n, n, order=4))
    g.init_taylor_green()
    g.set_diag_series(2)
    with pytest.raises(osb.OsbError) as e:
        osb.batch_step([g], 1)
    assert e.value.status == 2
    L = osb.load()
    assert L.osb_set_diag_series(g.handle, None, 0) == 0
    osb.batch_step([g], 1)

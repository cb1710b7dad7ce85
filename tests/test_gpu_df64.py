"""The double-float path (OSB_DF64) against the oracle, held to the FP64
path's bar: relative L2 per field <= 1e-12 for the residual and for states
after steps (Section 3.3 equations, Section 2.4 schemes)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs
from tests.helpers import conserved, rel_l2_fields

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def _grid(osb, nx, ny, nz, **kw):
    return osb.Grid(osb.Config(nx, ny, nz, precision=osb.OSB_DF64, **kw))


def _case(nx, ny, nz, **kw):
    return orc.Case(nx, ny, nz, **kw)


def _random_state(nx, ny, nz, seed):
    return conserved(*inputs.smooth_primitive_state(nx, ny, nz, seed), gamma=1.4)


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
@pytest.mark.parametrize("dims", [(16, 16, 16), (37, 20, 9)])
def test_df64_residual_matches_oracle(osb, order, dims):
    nx, ny, nz = dims
    Q = _random_state(nx, ny, nz, seed=order + nx)
    g = _grid(osb, nx, ny, nz, order=order, Re=100.0)
    g.set_state(Q)
    R = g.residual().cpu().numpy()
    Ro = orc.residual(_case(nx, ny, nz, order=order, Re=100.0), Q)
    errs = rel_l2_fields(R, Ro)
    print("df64 residual", order, dims, max(errs.values()))
    for m, err in errs.items():
        assert err < TOL, (m, err)


@pytest.mark.parametrize("n,order,steps", [(32, 4, 20), (8, 4, 10), (16, 6, 10), (24, 8, 8), (16, 12, 5)])
def test_df64_tgv_steps_match_oracle(osb, n, order, steps):
    g = _grid(osb, n, n, n, order=order)
    g.init_taylor_green()
    g.step(steps)
    case = _case(n, n, n, order=order)
    Qo = orc.rk3_step(case, orc.tgv_init(case), steps)
    errs = rel_l2_fields(g.get_state(), Qo)
    print("df64 steps", n, order, steps, max(errs.values()))
    for m, err in errs.items():
        assert err < TOL, (m, err)


def test_df64_noisy_noncubic_and_random_states(osb):
    nx, ny, nz = 40, 24, 18
    noise = inputs.gaussian_noise(nx, ny, nz, seed=1234)
    g = _grid(osb, nx, ny, nz, order=8, dt=1e-3)
    g.init_taylor_green(noise, 1e-4)
    g.step(6)
    case = _case(nx, ny, nz, order=8, dt=1e-3)
    Qo = orc.rk3_step(case, orc.tgv_init(case, noise, 1e-4), 6)
    for m, err in rel_l2_fields(g.get_state(), Qo).items():
        assert err < TOL, (m, err)
    Q = _random_state(20, 14, 11, seed=3)
    g = _grid(osb, 20, 14, 11, order=6, Re=200.0, dt=5e-4)
    g.set_state(Q)
    g.step(4)
    Qo = orc.rk3_step(_case(20, 14, 11, order=6, Re=200.0, dt=5e-4), Q, 4)
    for m, err in rel_l2_fields(g.get_state(), Qo).items():
        assert err < TOL, (m, err)


def test_df64_form_b_and_euler(osb):
    n = 16
    Q = _random_state(n, n, n, seed=21)
    g = _grid(osb, n, n, n, order=4, visc_form=osb.OSB_VISC_B, Re=300.0, dt=1e-3)
    g.set_state(Q)
    g.step(3)
    Qo = orc.rk3_step(_case(n, n, n, order=4, visc_form=1, Re=300.0, dt=1e-3), Q, 3)
    for m, err in rel_l2_fields(g.get_state(), Qo).items():
        assert err < TOL, (m, err)
    g = _grid(osb, n, n, n, order=4, dt=1e-3)
    g.set_state(Q)
    g.euler_step(2)
    g.step(2)
    case = _case(n, n, n, order=4, dt=1e-3)
    Qo = orc.rk3_step(case, orc.euler_step(case, Q, 2), 2)
    for m, err in rel_l2_fields(g.get_state(), Qo).items():
        assert err < TOL, (m, err)


def test_df64_conserves_totals(osb):
    n = 24
    g = _grid(osb, n, n, n, order=4, dt=2e-3)
    g.set_state(_random_state(n, n, n, seed=11))
    t0 = np.array(g.diagnostics()["total"])
    g.step(20)
    t1 = np.array(g.diagnostics()["total"])
    assert np.all(np.abs(t1 - t0) <= 1e-12 * np.maximum(np.abs(t0), 1.0))


def test_df64_graph_replay_equals_direct_launches(osb, monkeypatch):
    n = 16
    a = _grid(osb, n, n, n, order=4)
    a.init_taylor_green()
    a.step(4)                      # graph replay
    monkeypatch.setenv("OSB_GRAPHS", "0")
    b = _grid(osb, n, n, n, order=4)
    b.init_taylor_green()
    b.step(4)                      # direct launches
    assert np.array_equal(a.get_state(), b.get_state())


def test_df64_ensemble_equals_per_grid_steps(osb):
    """The ensemble's per-phase launches run the same double-float stage code."""
    specs = [(16, 800.0, 2e-3), (20, 1600.0, 1e-3), (12, 300.0, 3e-3)]
    a, b = [], []
    for i, (n, Re, dt) in enumerate(specs):
        for lst in (a, b):
            g = _grid(osb, n, n, n, order=4, Re=Re, dt=dt)
            g.init_taylor_green(inputs.gaussian_noise(n, n, n, 60 + i), 1e-3)
            lst.append(g)
    osb.batch_step(b, 3)
    for ga, gb, (n, Re, dt), i in zip(a, b, specs, range(3)):
        ga.step(3)
        A, B = ga.get_state(), gb.get_state()
        assert np.max(np.abs(A - B)) <= 1e-13 * np.max(np.abs(A))
        case = _case(n, n, n, order=4, Re=Re, dt=dt)
        Qo = orc.rk3_step(case, orc.tgv_init(case, inputs.gaussian_noise(n, n, n, 60 + i), 1e-3), 3)
        for m, err in rel_l2_fields(B, Qo).items():
            assert err < TOL, (m, err)


@pytest.mark.parametrize("mode", ["streams"])
def test_df64_ensemble_modes_match_persistent_kernel(osb, monkeypatch, mode):
    """Concurrent-stream step graphs (the double-float default) against the
    persistent kernel (OSB_BATCH_MODE) on uneven grids, ragged in y (extents
    not multiples of the 8-row tile), over two calls with different parities;
    the stream mode replays the per-grid step graphs, so it also equals
    per-grid stepping bit for bit."""
    specs = [(16, 800.0, 2e-3), (20, 1600.0, 1e-3), (12, 300.0, 3e-3), (28, 500.0, 1.5e-3)]
    runs = []
    for m in ("persistent", mode, "single"):
        monkeypatch.setenv("OSB_BATCH_MODE", m)
        gs = []
        for i, (n, Re, dt) in enumerate(specs):
            g = _grid(osb, n, n + 2, n, order=4, Re=Re, dt=dt)
            g.init_taylor_green(inputs.gaussian_noise(n, n + 2, n, 80 + i), 1e-3)
            gs.append(g)
        if m == "single":
            for g in gs:
                g.step(5)
        else:
            osb.batch_step(gs, 3)
            osb.batch_step(gs, 2)
        runs.append([g.get_state() for g in gs])
    for A, B, C in zip(*runs):
        assert np.max(np.abs(A - B)) <= 1e-13 * np.max(np.abs(A))
        if mode == "streams":
            assert np.array_equal(B, C)

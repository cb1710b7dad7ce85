"""Ensemble stepping: one persistent, graph-captured launch over grids of
uneven sizes and parameters (osb_batch_step), its bounded waits, and the
tile autotuner."""
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
    m.batch_configure(2.0, False)
    return m


@pytest.fixture(autouse=True)
def persistent_kernel(monkeypatch):
    """These tests cover the persistent kernel's work items unless a test
    picks another mode itself.  Its FP32 z-march items run the 32x8 residual
    kernel at every order, so the per-grid steps they are compared with do too
    (orders 6 and 8 default to the narrow kernel, whose z sums are added in
    another order)."""
    monkeypatch.setenv("OSB_BATCH_MODE", "persistent")
    monkeypatch.setenv("OSB_FP32_ZRHS", "wide")


def _ensemble(osb, specs, precision, order=4, seed=3):
    grids = []
    for i, (n, Re, M, dt) in enumerate(specs):
        g = osb.Grid(osb.Config(n, n, n, order=order, precision=precision, Re=Re, Mach=M, dt=dt))
        g.init_taylor_green(inputs.gaussian_noise(n, n, n, seed + i), 1e-3)
        grids.append(g)
    return grids


def _assert_fp32_instantiations_agree(A, B, tag=None):
    """The ensemble kernel and the per-grid kernels run the same z-march code,
    but the compiler may pair multiplies and adds into FMAs differently in the
    two instantiations: the states agree to a few FP32 roundings of the stage
    residual (relative 1e-7), far below the FP32 bound against the oracle
    (1e-5) and far below what a stale or racing read would leave (>= 1e-4)."""
    mnorm = np.linalg.norm(A[1:4].ravel())
    for m in range(5):
        scale = mnorm if 1 <= m <= 3 else np.linalg.norm(A[m].ravel())
        assert np.linalg.norm((A[m] - B[m]).ravel()) / scale < 1e-7, (tag, m)


SPECS = [(16, 1600.0, 0.1, 2e-3), (24, 400.0, 0.2, 1.5e-3), (12, 3000.0, 0.05, 3e-3), (20, 100.0, 0.3, 1e-3)]


def test_batch_equals_per_grid_steps_bitwise_fp64(osb):
    a = _ensemble(osb, SPECS, osb.OSB_FP64)
    b = _ensemble(osb, SPECS, osb.OSB_FP64)
    for g in a:
        g.step(7)
    osb.batch_step(b, 3)      # odd count: the register roles flip
    osb.batch_step(b, 4)      # different parity pattern, new graph
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.get_state(), gb.get_state())
        assert gb.diagnostics()["step"] == 7


def test_batch_graph_replay_and_mixed_parity(osb):
    a = _ensemble(osb, SPECS, osb.OSB_FP64)
    b = _ensemble(osb, SPECS, osb.OSB_FP64)
    b[1].step(1)              # instances start with different register parities
    a[1].step(1)
    for _ in range(3):
        osb.batch_step(b, 2)  # same key: the captured graph is replayed
    for g in a:
        g.step(6)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.get_state(), gb.get_state())


@pytest.mark.parametrize("order", [4, 8])
def test_batch_fp32_close_to_oracle(osb, order):
    specs = [(16, 800.0, 0.15, 2e-3), (24, 1600.0, 0.1, 1e-3)]
    grids = _ensemble(osb, specs, osb.OSB_FP32, order=order, seed=11)
    osb.batch_step(grids, 6)
    for i, ((n, Re, M, dt), g) in enumerate(zip(specs, grids)):
        case = orc.Case(n, n, n, order=order, Re=Re, Mach=M, dt=dt)
        Qo = orc.rk3_step(case, orc.tgv_init(case, inputs.gaussian_noise(n, n, n, 11 + i), 1e-3), 6)
        Q = g.get_state()
        mnorm = np.linalg.norm(Qo[1:4].ravel())
        for m in range(5):
            scale = mnorm if 1 <= m <= 3 else np.linalg.norm(Qo[m].ravel())
            assert np.linalg.norm((Q[m] - Qo[m]).ravel()) / scale < 1e-5


def test_batch_fp32_zmarch_items_match_per_grid_steps(osb, monkeypatch):
    """FP32 ensembles whose x extents are multiples of 4 run z-march items in
    the persistent kernel; per point they do the arithmetic of the per-grid
    z-march stage (ragged x and y tiles included)."""
    monkeypatch.setenv("OSB_FP32_STAGE", "zmarch")
    specs = [(20, 1600.0, 0.1, 2e-3), (36, 400.0, 0.2, 1.5e-3), (12, 3000.0, 0.05, 3e-3), (32, 100.0, 0.3, 1e-3)]
    for order in (2, 4, 6, 8):
        a = _ensemble(osb, specs, osb.OSB_FP32, order=order, seed=31)
        b = _ensemble(osb, specs, osb.OSB_FP32, order=order, seed=31)
        for g in a:
            g.step(5)
        osb.batch_step(b, 2)
        osb.batch_step(b, 3)
        for ga, gb in zip(a, b):
            _assert_fp32_instantiations_agree(ga.get_state(), gb.get_state(), order)
            assert gb.diagnostics()["step"] == 5


def test_batch_fp32_zmarch_items_with_tma_tiles(osb, monkeypatch):
    """Grids wide enough for interior tiles (x >= 72, y >= 18): the persistent
    kernel loads their planes with TMA boxes whose descriptors live in the
    device record; results agree with per-grid stepping and the oracle."""
    monkeypatch.setenv("OSB_FP32_STAGE", "zmarch")
    specs = [(72, 24, 16), (104, 32, 12)]
    grids, refs = [], []
    for i, (nx, ny, nz) in enumerate(specs):
        noise = inputs.gaussian_noise(nx, ny, nz, 51 + i)
        g = osb.Grid(osb.Config(nx, ny, nz, order=4, precision=osb.OSB_FP32, dt=2e-3))
        g.init_taylor_green(noise, 1e-3)
        r = osb.Grid(osb.Config(nx, ny, nz, order=4, precision=osb.OSB_FP32, dt=2e-3))
        r.init_taylor_green(noise, 1e-3)
        grids.append(g)
        refs.append(r)
    osb.batch_step(grids, 3)
    for (nx, ny, nz), i, g, r in zip(specs, range(2), grids, refs):
        r.step(3)
        _assert_fp32_instantiations_agree(r.get_state(), g.get_state(), (nx, ny, nz))
        case = orc.Case(nx, ny, nz, order=4, dt=2e-3)
        Qo = orc.rk3_step(case, orc.tgv_init(case, inputs.gaussian_noise(nx, ny, nz, 51 + i), 1e-3), 3)
        Q = g.get_state()
        mnorm = np.linalg.norm(Qo[1:4].ravel())
        for m in range(5):
            scale = mnorm if 1 <= m <= 3 else np.linalg.norm(Qo[m].ravel())
            assert np.linalg.norm((Q[m] - Qo[m]).ravel()) / scale < 1e-5


def test_batch_steps_mix_with_fused_per_grid_steps(osb):
    """Per-grid FP32 steps of orders 2 and 4 run the fused stage, whose
    stage registers differ from the ensemble's z-march items only inside a
    step: steps of either kind may follow each other on the same grids.  The
    mixed sequence agrees with per-grid steps to FP32 rounding of the stage
    residuals, and with the oracle within the FP32 bound."""
    specs = [(24, 800.0, 0.15, 2e-3), (32, 1600.0, 0.1, 1e-3)]
    for order in (2, 4):
        a = _ensemble(osb, specs, osb.OSB_FP32, order=order, seed=61)
        b = _ensemble(osb, specs, osb.OSB_FP32, order=order, seed=61)
        for g in a:
            g.step(6)
        for g in b:
            g.step(2)
        osb.batch_step(b, 2)
        for g in b:
            g.step(2)
        for i, (ga, gb) in enumerate(zip(a, b)):
            A, B = ga.get_state(), gb.get_state()
            mnorm = np.linalg.norm(A[1:4].ravel())
            for m in range(5):
                scale = mnorm if 1 <= m <= 3 else np.linalg.norm(A[m].ravel())
                assert np.linalg.norm((A[m] - B[m]).ravel()) / scale < 2e-6, (order, i, m)
            n, Re, M, dt = specs[i]
            case = orc.Case(n, n, n, order=order, Re=Re, Mach=M, dt=dt)
            Qo = orc.rk3_step(case, orc.tgv_init(case, inputs.gaussian_noise(n, n, n, 61 + i), 1e-3), 6)
            mo = np.linalg.norm(Qo[1:4].ravel())
            for m in range(5):
                scale = mo if 1 <= m <= 3 else np.linalg.norm(Qo[m].ravel())
                assert np.linalg.norm((B[m] - Qo[m]).ravel()) / scale < 1e-5, (order, i, m)


def test_batch_fp32_unaligned_extent_uses_point_items(osb):
    """An x extent that is not a multiple of 4 sends the whole FP32 ensemble to
    the three-kernel items; the result still meets the FP32 bound."""
    specs = [(18, 800.0, 0.15, 2e-3), (16, 1600.0, 0.1, 1e-3)]
    grids = _ensemble(osb, specs, osb.OSB_FP32, order=4, seed=41)
    osb.batch_step(grids, 4)
    for i, ((n, Re, M, dt), g) in enumerate(zip(specs, grids)):
        case = orc.Case(n, n, n, order=4, Re=Re, Mach=M, dt=dt)
        Qo = orc.rk3_step(case, orc.tgv_init(case, inputs.gaussian_noise(n, n, n, 41 + i), 1e-3), 4)
        Q = g.get_state()
        mnorm = np.linalg.norm(Qo[1:4].ravel())
        for m in range(5):
            scale = mnorm if 1 <= m <= 3 else np.linalg.norm(Qo[m].ravel())
            assert np.linalg.norm((Q[m] - Qo[m]).ravel()) / scale < 1e-5


def test_batch_fp64_matches_oracle(osb):
    specs = [(12, 500.0, 0.2, 2e-3), (16, 1600.0, 0.1, 2e-3)]
    grids = _ensemble(osb, specs, osb.OSB_FP64, order=6, seed=21)
    osb.batch_step(grids, 3)
    for i, ((n, Re, M, dt), g) in enumerate(zip(specs, grids)):
        case = orc.Case(n, n, n, order=6, Re=Re, Mach=M, dt=dt)
        Qo = orc.rk3_step(case, orc.tgv_init(case, inputs.gaussian_noise(n, n, n, 21 + i), 1e-3), 3)
        Q = g.get_state()
        for m in range(5):
            assert np.linalg.norm(Q[m] - Qo[m]) / np.linalg.norm(Qo[m]) < 1e-12


def test_batch_wait_limit_reports_timeout_and_context_survives(osb):
    """A wait on a count that nothing reaches runs out after its limit: the call
    returns OSB_ERR_TIMEOUT (no trap, no hang) and the GPU keeps working."""
    grids = _ensemble(osb, SPECS[:2], osb.OSB_FP64)
    osb.batch_configure(0.05, True)
    try:
        with pytest.raises(osb.OsbError) as ei:
            osb.batch_step(grids, 2)
        assert ei.value.status == 5
    finally:
        osb.batch_configure(2.0, False)
    fresh = _ensemble(osb, SPECS[:2], osb.OSB_FP64)
    ref = _ensemble(osb, SPECS[:2], osb.OSB_FP64)
    osb.batch_step(fresh, 2)
    for g in ref:
        g.step(2)
    for a, b in zip(fresh, ref):
        assert np.array_equal(a.get_state(), b.get_state())


def test_batch_fp32_zmarch_wait_limit_reports_timeout(osb):
    grids = _ensemble(osb, [(16, 1600.0, 0.1, 2e-3), (24, 400.0, 0.2, 1e-3)], osb.OSB_FP32)
    osb.batch_configure(0.05, True)
    try:
        with pytest.raises(osb.OsbError) as ei:
            osb.batch_step(grids, 2)
        assert ei.value.status == 5
    finally:
        osb.batch_configure(2.0, False)
    fresh = _ensemble(osb, [(16, 1600.0, 0.1, 2e-3)], osb.OSB_FP32)
    ref = _ensemble(osb, [(16, 1600.0, 0.1, 2e-3)], osb.OSB_FP32)
    osb.batch_step(fresh, 2)
    ref[0].step(2)
    _assert_fp32_instantiations_agree(ref[0].get_state(), fresh[0].get_state())


def test_batch_rejects_mixed_configurations(osb):
    a = osb.Grid(osb.Config(8, 8, 8, order=4))
    b = osb.Grid(osb.Config(8, 8, 8, order=8))
    with pytest.raises(osb.OsbError) as ei:
        osb.batch_step([a, b], 1)
    assert ei.value.status == 2
    with pytest.raises(osb.OsbError):
        osb.batch_step([a, a], 1)


def test_autotune_restores_state(osb, tmp_path, monkeypatch):
    g = _ensemble(osb, [(24, 1600.0, 0.1, 1e-3)], osb.OSB_FP64)[0]
    g.step(2)
    before = g.get_state()
    d0 = g.diagnostics()
    tz = osb.autotune(g, trial_steps=2)
    assert tz in (1, 2, 4, 8, 16)
    assert np.array_equal(g.get_state(), before)
    d1 = g.diagnostics()
    assert d1["step"] == d0["step"] and d1["t"] == d0["t"]
    g.step(1)  # still usable


def test_autotune_fp32_candidates(osb):
    g = _ensemble(osb, [(32, 1600.0, 0.1, 1e-3)], osb.OSB_FP32)[0]
    before = g.get_state()
    tz = osb.autotune(g, trial_steps=2)
    assert tz in (4, 8, 16, 32)
    assert np.array_equal(g.get_state(), before)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_stream_mode_equals_per_grid_steps_bitwise(osb, monkeypatch, precision):
    """OSB_BATCH_MODE=streams replays each grid's own step graph on one of the
    library's concurrent streams: bit for bit the per-grid steps, over calls
    with odd and even step counts (the grids' register roles flip)."""
    prec = osb.OSB_FP64 if precision == "fp64" else osb.OSB_FP32
    a = _ensemble(osb, SPECS, prec)
    b = _ensemble(osb, SPECS, prec)
    for g in a:
        g.step(6)
    monkeypatch.setenv("OSB_BATCH_MODE", "streams")
    osb.batch_step(b, 1)
    osb.batch_step(b, 3)
    osb.batch_step(b, 2)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.get_state(), gb.get_state())


def test_batch_stream_mode_more_grids_than_streams(osb, monkeypatch):
    """Twelve grids on the 8 library streams (some streams replay several
    grids' step graphs in turn): bit for bit the per-grid steps."""
    specs = [(8 + 2 * (i % 5), 200.0 + 150.0 * i, 0.1 + 0.01 * i, 1e-3 + 1e-4 * (i % 3)) for i in range(12)]
    a = _ensemble(osb, specs, osb.OSB_FP64, seed=40)
    b = _ensemble(osb, specs, osb.OSB_FP64, seed=40)
    for g in a:
        g.step(3)
    monkeypatch.setenv("OSB_BATCH_MODE", "streams")
    osb.batch_step(b, 3)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.get_state(), gb.get_state())


def test_batch_autotune_restores_states_and_sets_depths(osb):
    """The in-ensemble tuner times candidate depths on the whole ensemble and
    restores every grid: stepping afterwards equals stepping untouched grids,
    and every shape's depth is one of the candidates."""
    specs = [(16, 1600.0, 0.1, 2e-3), (24, 400.0, 0.2, 1.5e-3), (16, 800.0, 0.15, 2e-3), (32, 100.0, 0.3, 1e-3)]
    for prec, cands in ((osb.OSB_FP32, {4, 8, 16, 32}), (osb.OSB_FP64, {1, 2, 4, 8, 16})):
        a = _ensemble(osb, specs, prec, seed=50)
        b = _ensemble(osb, specs, prec, seed=50)
        depths = osb.autotune_batch(b, trial_steps=1)
        assert set(depths) == {(16, 16, 16), (24, 24, 24), (32, 32, 32)}
        assert all(v in cands for v in depths.values()), depths
        for g in b:
            assert g.diagnostics()["step"] == 0
        osb.batch_step(a, 3)
        osb.batch_step(b, 3)
        for ga, gb in zip(a, b):
            assert np.array_equal(ga.get_state(), gb.get_state())


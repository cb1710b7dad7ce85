"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances: FP64 results must match the oracle to a relative L2 of 1e-12 per
field after N steps (the bar of the FP64 path).  The residual itself is held
to the same 1e-12.  The FP32 path is held to a bound derived from FP32
rounding (see test_fp32_*).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs
from tests.helpers import conserved, rel_l2, rel_l2_fields

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


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
    return osb.Grid(osb.Config(nx, ny, nz, **kw))


def _case(nx, ny, nz, **kw):
    kw = {k: v for k, v in kw.items() if k != "precision"}
    return orc.Case(nx, ny, nz, **kw)


def _random_state(nx, ny, nz, seed, gamma=1.4):
    return conserved(*inputs.smooth_primitive_state(nx, ny, nz, seed), gamma=gamma)


# --------------------------------------------------------------------------
def test_initial_state_matches_oracle(osb):
    for (nx, ny, nz) in [(8, 8, 8), (32, 32, 32), (17, 12, 9)]:
        g = _grid(osb, nx, ny, nz)
        g.init_taylor_green()
        Q = g.get_state()
        Qo = orc.tgv_init(_case(nx, ny, nz))
        assert rel_l2(Q, Qo) < 4e-15
        noise = inputs.gaussian_noise(nx, ny, nz, seed=1234)
        g.init_taylor_green(noise, 1e-4)
        Qo = orc.tgv_init(_case(nx, ny, nz), noise, 1e-4)
        assert rel_l2(g.get_state(), Qo) < 4e-15


@pytest.mark.parametrize("n,order", [(32, 4), (8, 4), (24, 8), (16, 2)])
def test_initial_diagnostics_closed_form(osb, n, order):
    g = _grid(osb, n, n, n, order=order)
    g.init_taylor_green()
    dg = g.diagnostics()
    c, _ = orc.fd_coeffs(order)
    h = 2 * math.pi / n
    k1 = sum(2 * c[m] * math.sin(m * h) for m in range(1, order // 2 + 1)) / h
    gM2 = 1.4 * 0.01
    assert dg["ke"] == pytest.approx(0.125, rel=1e-13)
    assert dg["enstrophy"] == pytest.approx(k1 ** 2 * (3 / 8 - 5 * gM2 / 128), rel=1e-13)
    assert dg["total"][0] == pytest.approx(1.0, rel=1e-13)
    assert dg["nonfinite"] == 0


def test_diagnostics_match_oracle_on_random_state(osb):
    nx, ny, nz = 20, 14, 11
    Q = _random_state(nx, ny, nz, seed=9)
    g = _grid(osb, nx, ny, nz, order=6, dt=1e-3)
    g.set_state(Q)
    dg = g.diagnostics()
    do = orc.diagnostics(_case(nx, ny, nz, order=6, dt=1e-3), Q)
    assert dg["ke"] == pytest.approx(do["ke"], rel=1e-13)
    assert dg["enstrophy"] == pytest.approx(do["enstrophy"], rel=1e-13)
    for m, k in enumerate(("rho", "rhou0", "rhou1", "rhou2", "rhoE")):
        assert dg["total"][m] == pytest.approx(do[k], rel=1e-12, abs=1e-15)
    assert dg["max_cfl"] == pytest.approx(do["max_cfl"], rel=1e-13)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
@pytest.mark.parametrize("dims", [(16, 16, 16), (37, 20, 9), (8, 8, 8)])
def test_residual_matches_oracle(osb, order, dims):
    """Several 32x8 tiles plus ragged tails in x and y; 8^3 wraps the widest
    stencils around the box."""
    nx, ny, nz = dims
    Q = _random_state(nx, ny, nz, seed=order + nx)
    g = _grid(osb, nx, ny, nz, order=order, Re=100.0)
    g.set_state(Q)
    R = g.residual().cpu().numpy()
    Ro = orc.residual(_case(nx, ny, nz, order=order, Re=100.0), Q)
    for m, err in rel_l2_fields(R, Ro).items():
        assert err < TOL64, (m, err)


@pytest.mark.parametrize("n,order,steps", [(32, 4, 20), (8, 4, 10), (8, 8, 10), (16, 6, 10), (48, 8, 5)])
def test_tgv_steps_match_oracle(osb, n, order, steps):
    """The small Taylor-Green case (32^3, 4th order, 20 steps of dt = 3.385e-3)
    and variants: rel-L2 per field <= 1e-12."""
    g = _grid(osb, n, n, n, order=order)
    g.init_taylor_green()
    g.step(steps)
    Q = g.get_state()
    case = _case(n, n, n, order=order)
    Qo = orc.rk3_step(case, orc.tgv_init(case), steps)
    for m, err in rel_l2_fields(Q, Qo).items():
        assert err < TOL64, (m, err)


def test_noisy_nonCubic_steps_match_oracle(osb):
    nx, ny, nz = 40, 24, 18
    noise = inputs.gaussian_noise(nx, ny, nz, seed=1234)
    g = _grid(osb, nx, ny, nz, order=8, dt=1e-3)
    g.init_taylor_green(noise, 1e-4)
    g.step(6)
    case = _case(nx, ny, nz, order=8, dt=1e-3)
    Qo = orc.rk3_step(case, orc.tgv_init(case, noise, 1e-4), 6)
    for m, err in rel_l2_fields(g.get_state(), Qo).items():
        assert err < TOL64, (m, err)


def test_random_state_steps_match_oracle(osb):
    nx, ny, nz = 24, 16, 20
    Q0 = _random_state(nx, ny, nz, seed=5)
    g = _grid(osb, nx, ny, nz, order=4, Re=50.0, dt=1e-3)
    g.set_state(Q0)
    g.step(4)
    Qo = orc.rk3_step(_case(nx, ny, nz, order=4, Re=50.0, dt=1e-3), Q0, 4)
    for m, err in rel_l2_fields(g.get_state(), Qo).items():
        assert err < TOL64, (m, err)


@pytest.mark.parametrize("order", [2, 4, 8])
def test_form_b_residual_matches_oracle(osb, order):
    """Viscous work by the product rule (form B): u_i d_j tau_ij + tau_ij d_j u_i."""
    nx, ny, nz = 33, 18, 12
    Q = _random_state(nx, ny, nz, seed=40 + order)
    g = _grid(osb, nx, ny, nz, order=order, visc_form=osb.OSB_VISC_B, Re=30.0)
    g.set_state(Q)
    R = g.residual().cpu().numpy()
    Ro = orc.residual(_case(nx, ny, nz, order=order, visc_form=1, Re=30.0), Q)
    for m, err in rel_l2_fields(R, Ro).items():
        assert err < TOL64, (m, err)


def test_form_b_steps_match_oracle(osb):
    n = 24
    noise = inputs.gaussian_noise(n, n, n, seed=8)
    g = _grid(osb, n, n, n, order=4, visc_form=osb.OSB_VISC_B)
    g.init_taylor_green(noise, 1e-3)
    g.step(8)
    case = _case(n, n, n, order=4, visc_form=1)
    Qo = orc.rk3_step(case, orc.tgv_init(case, noise, 1e-3), 8)
    for m, err in rel_l2_fields(g.get_state(), Qo).items():
        assert err < TOL64, (m, err)


# --------------------------------------------------------------------------
def test_conservation_on_gpu(osb):
    n = 32
    g = _grid(osb, n, n, n, order=8)
    noise = inputs.gaussian_noise(n, n, n, seed=3)
    g.init_taylor_green(noise, 1e-2)
    d0 = g.diagnostics()
    g.step(30)
    d1 = g.diagnostics()
    for m in range(5):
        scale = max(abs(d0["total"][m]), 1.0)
        assert abs(d1["total"][m] - d0["total"][m]) < 1e-13 * 30 * 3 * scale


def test_checkpoint_restart_is_bitwise(osb):
    n = 16
    a = _grid(osb, n, n, n)
    a.init_taylor_green()
    a.step(6)
    full = a.get_state()
    b = _grid(osb, n, n, n)
    b.init_taylor_green()
    b.step(3)
    mid = b.get_state()
    c = _grid(osb, n, n, n)
    c.set_state(mid)
    c.step(3)
    assert np.array_equal(c.get_state(), full)


def test_runs_are_deterministic(osb):
    n = 24
    out = []
    for _ in range(2):
        g = _grid(osb, n, n, n, order=4)
        g.init_taylor_green(inputs.gaussian_noise(n, n, n, seed=2), 1e-3)
        g.step(5)
        out.append((g.get_state(), g.diagnostics()))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1]["ke"] == out[1][1]["ke"] and out[0][1]["enstrophy"] == out[1][1]["enstrophy"]


def test_nonfinite_state_is_reported(osb):
    n = 8
    g = _grid(osb, n, n, n)
    Q = orc.tgv_init(_case(n, n, n))
    Q[3, 1, 2, 3] = np.nan
    g.set_state(Q)
    dg = g.diagnostics(raise_nonfinite=False)
    assert dg["status"] == 4 and dg["nonfinite"] == 1
    with pytest.raises(osb.OsbError):
        g.diagnostics()


def test_batch_step_matches_single_grids(osb):
    sizes = [(16, 16, 16, 1600.0, 0.1), (24, 24, 24, 400.0, 0.2), (12, 12, 12, 3000.0, 0.05)]
    singles, batch = [], []
    for (nx, ny, nz, Re, M) in sizes:
        for lst in (singles, batch):
            g = _grid(osb, nx, ny, nz, Re=Re, Mach=M, dt=1e-3)
            g.init_taylor_green()
            lst.append(g)
    for g in singles:
        g.step(4)
    osb.batch_step(batch, 4)
    for a, b in zip(singles, batch):
        assert np.array_equal(a.get_state(), b.get_state())


# --------------------------------------------------------------------------
# FP32 path: stencils in FP32, U accumulator and reductions in FP64
# --------------------------------------------------------------------------
@pytest.mark.parametrize("order", [4, 8])
def test_fp32_residual_error_is_fp32_rounding(osb, order):
    """FP32 residual vs the FP64 oracle: the error is FP32 rounding of the
    inputs and intermediates amplified by the stencil cancellation (~1/h),
    so rel-L2 stays below ~1e3 * 2^-24 at these sizes."""
    n = 24
    Q = _random_state(n, n, n, seed=17)
    g = _grid(osb, n, n, n, order=order, precision=osb.OSB_FP32, Re=100.0)
    g.set_state(Q)
    R = g.residual().cpu().numpy()
    Ro = orc.residual(_case(n, n, n, order=order, Re=100.0), Q)
    for m, err in rel_l2_fields(R, Ro).items():
        assert err < 1e3 * 2.0 ** -24, (m, err)


def test_fp32_tgv_steps_close_to_oracle(osb):
    """FP32 stencils, FP64 accumulator, 20 steps of the small Taylor-Green case.
    Each stage rounds q to FP32 (2^-24) and evaluates R in FP32; the stencil
    cancellation amplifies that by ~|Q|/(h |dQ/dx|) (<= ~1e2 for rho E ~ 178
    carrying O(1) fluctuations), and the errors enter U once per stage times dt:
    after t = 0.068 the error is ~ t * |R| * 1e2 * 2^-24 ~ 1e-6 of |Q|.  Momentum
    components are measured against the momentum magnitude (rho u2 starts at
    exactly zero, so its own norm is no scale); bound 1e-5."""
    n, steps = 32, 20
    g = _grid(osb, n, n, n, order=4, precision=osb.OSB_FP32)
    g.init_taylor_green()
    g.step(steps)
    Q = g.get_state()
    case = _case(n, n, n, order=4)
    Qo = orc.rk3_step(case, orc.tgv_init(case), steps)
    mnorm = np.linalg.norm(Qo[1:4].ravel())
    for m in range(5):
        scale = mnorm if 1 <= m <= 3 else np.linalg.norm(Qo[m].ravel())
        err = np.linalg.norm((Q[m] - Qo[m]).ravel()) / scale
        assert err < 1e-5, (m, err)


def _fp32_err(Q, Qo):
    """Per-field error of an FP32-path state: momentum components against the
    momentum magnitude, the others against their own norm."""
    mnorm = np.linalg.norm(Qo[1:4].ravel())
    out = []
    for m in range(5):
        scale = mnorm if 1 <= m <= 3 else np.linalg.norm(Qo[m].ravel())
        out.append(np.linalg.norm((Q[m] - Qo[m]).ravel()) / scale)
    return out


@pytest.mark.parametrize("dims,order", [((32, 32, 32), 4), ((40, 24, 48), 8), ((8, 8, 8), 8),
                                        ((37, 20, 9), 2), ((24, 16, 40), 6), ((70, 9, 33), 4)])
def test_fp32_zmarch_steps_close_to_oracle(osb, dims, order):
    """The z-marching FP32 stage (tiles of 32x8 columns, 32-plane z chunks,
    ragged tiles, nz below the stencil width) against the FP64 oracle, with
    the FP32 bound derived in test_fp32_tgv_steps_close_to_oracle."""
    nx, ny, nz = dims
    steps = 10
    noise = inputs.gaussian_noise(nx, ny, nz, seed=77)
    g = _grid(osb, nx, ny, nz, order=order, precision=osb.OSB_FP32, dt=2e-3, Re=200.0)
    g.init_taylor_green(noise, 1e-2)
    g.step(steps)
    case = _case(nx, ny, nz, order=order, dt=2e-3, Re=200.0)
    Qo = orc.rk3_step(case, orc.tgv_init(case, noise, 1e-2), steps)
    for m, err in enumerate(_fp32_err(g.get_state(), Qo)):
        assert err < 1e-5, (m, err)


@pytest.mark.parametrize("order", [4, 8])
def test_fp32_zmarch_agrees_with_three_kernel_stage(osb, order, monkeypatch):
    """The two FP32 stage implementations evaluate the same discrete operator:
    their states after 5 steps differ only by FP32 rounding."""
    n = 40
    noise = inputs.gaussian_noise(n, n, n, seed=5)
    out = []
    for mode in ("zmarch", "split3"):
        monkeypatch.setenv("OSB_FP32_STAGE", mode)
        g = _grid(osb, n, n, n, order=order, precision=osb.OSB_FP32)
        g.init_taylor_green(noise, 1e-3)
        g.step(5)
        out.append(g.get_state())
    for m, err in enumerate(_fp32_err(out[0], out[1])):
        assert err < 2e-6, (m, err)


@pytest.mark.parametrize("dims,order", [((36, 18, 20), 8), ((30, 14, 11), 8), ((72, 22, 9), 6), ((8, 6, 5), 6)])
def test_fp32_narrow_residual_kernel_agrees_with_wide_one(osb, dims, order, monkeypatch):
    """Orders 6 and 8 take the narrow residual kernel (32x4 tiles, z taps of
    the flux and viscous sums scattered into pending sums); OSB_FP32_ZRHS=wide
    the 32x8 one with register queues.  Same operator, other summation order:
    the states after five steps differ by FP32 rounding only.  y extents not a
    multiple of 4 (ragged narrow tiles), an x extent that is not a multiple of 4
    (4-byte loads), and a grid smaller than the stencil are included."""
    nx, ny, nz = dims
    noise = inputs.gaussian_noise(nx, ny, nz, seed=15)
    out = []
    for mode in ("narrow", "wide"):
        monkeypatch.setenv("OSB_FP32_ZRHS", mode)
        g = _grid(osb, nx, ny, nz, order=order, precision=osb.OSB_FP32, dt=1e-3, Re=400.0)
        g.init_taylor_green(noise, 1e-2)
        g.step(5)
        out.append(g.get_state())
        assert g.diagnostics()["nonfinite"] == 0
    for m, err in enumerate(_fp32_err(out[0], out[1])):
        assert err < 2e-6, (m, err)


@pytest.mark.parametrize("dims,order", [((40, 40, 40), 4), ((72, 20, 30), 4), ((37, 20, 9), 2), ((64, 24, 17), 2),
                                        ((70, 9, 33), 4), ((6, 5, 3), 4)])
def test_fp32_fused_stage_agrees_with_two_and_three_kernel_stages(osb, dims, order, monkeypatch):
    """The fused FP32 stage (one kernel per RK stage, FP32 increments in stages
    1-2 and one FP64 accumulation per step) evaluates the same discrete
    operator as the two z-march kernels and the three-kernel stage: after five
    steps the states differ by FP32 rounding only.  Ragged tiles, odd and
    non-multiple-of-4 x extents (scalar and 4-byte loads) and a grid smaller
    than the stencil in every direction are included."""
    nx, ny, nz = dims
    noise = inputs.gaussian_noise(nx, ny, nz, seed=5)
    out = {}
    for mode in ("fused", "zmarch", "split3"):
        monkeypatch.setenv("OSB_FP32_STAGE", mode)
        g = _grid(osb, nx, ny, nz, order=order, precision=osb.OSB_FP32)
        g.init_taylor_green(noise, 1e-3)
        g.step(5)
        out[mode] = g.get_state()
        assert g.diagnostics()["nonfinite"] == 0
    for other in ("zmarch", "split3"):
        for m, err in enumerate(_fp32_err(out["fused"], out[other])):
            assert err < 2e-6, (other, m, err)


@pytest.mark.parametrize("order", [2, 4])
def test_fp32_fused_stage_independent_of_work_split(osb, order, monkeypatch):
    """The fused stage's CTAs each march a contiguous run of the (tile, z)
    planes, restarting with warm-up planes wherever a run enters a new tile.
    Every output point sees the same operands, summed in the same order, however
    the runs fall, so one CTA (every tile in turn), seven CTAs (runs that cross
    tile boundaries mid-column) and the default split give the same state bit
    for bit."""
    nx, ny, nz = 64, 16, 23
    noise = inputs.gaussian_noise(nx, ny, nz, seed=9)
    outs = []
    for ctas in ("1", "7", None):
        if ctas is None:
            monkeypatch.delenv("OSB_FUSED_CTAS", raising=False)
        else:
            monkeypatch.setenv("OSB_FUSED_CTAS", ctas)
        g = _grid(osb, nx, ny, nz, order=order, precision=osb.OSB_FP32, dt=2e-3)
        g.init_taylor_green(noise, 1e-2)
        g.step(3)
        outs.append(g.get_state())
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("dims,order", [((128, 24, 40), 4), ((104, 32, 20), 8), ((112, 40, 12), 6),
                                        ((96, 40, 20), 2)])
def test_fp32_tma_and_cpasync_loads_are_bitwise_equal(osb, dims, order, monkeypatch):
    """Grids wide enough for interior tiles: those load planes with TMA boxes,
    boundary tiles with wrapped cp.async copies.  Both fill shared memory with
    the same values, so the states agree bitwise with the all-cp.async run, and
    both stay within the FP32 bound of the oracle."""
    nx, ny, nz = dims
    noise = inputs.gaussian_noise(nx, ny, nz, seed=31)
    out = []
    for mode in ("tma", "cpasync"):
        monkeypatch.setenv("OSB_FP32_LOADS", mode)
        g = _grid(osb, nx, ny, nz, order=order, precision=osb.OSB_FP32, dt=1e-3, Re=400.0)
        g.init_taylor_green(noise, 1e-2)
        g.step(4)
        out.append(g.get_state())
        assert g.diagnostics()["nonfinite"] == 0
    assert np.array_equal(out[0], out[1])
    case = _case(nx, ny, nz, order=order, dt=1e-3, Re=400.0)
    Qo = orc.rk3_step(case, orc.tgv_init(case, noise, 1e-2), 4)
    for m, err in enumerate(_fp32_err(out[0], Qo)):
        assert err < 1e-5, (m, err)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replayed_steps_equal_direct_launches(osb, precision, monkeypatch):
    """Multi-step calls replay a captured CUDA graph of one step; the state is
    bitwise the one of direct launches (one call per step)."""
    n = 24
    noise = inputs.gaussian_noise(n, n, n, seed=41)
    a = _grid(osb, n, n, n, order=4, precision=precision)
    b = _grid(osb, n, n, n, order=4, precision=precision)
    a.init_taylor_green(noise, 1e-3)
    b.init_taylor_green(noise, 1e-3)
    a.step(7)
    for _ in range(7):
        b.step(1)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.diagnostics()["step"] == 7

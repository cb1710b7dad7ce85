"""Symmetry boundaries (Section 2.6) on the GPU, through the C ABI, against the
oracle (the periodic scheme on the mirror-extended grid, restricted).

FP64 and double-float: relative L2 per field 1e-12 (residual and steps);
FP32: 1e-5 (its rounding bound, as for periodic grids).  Every symmetric
pattern of axes, both viscous forms, orders 2 to 12, extents below the
stencil radius (multiple mirrorings), the Taylor-Green octant against the
GPU's own periodic run of the full box, diagnostics, the forward Euler step,
and the calls that refuse symmetric grids.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs
from tests.helpers import conserved, rel_l2, rel_l2_fields

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 2: 1e-12, 1: 1e-5}  # OSB_FP64, OSB_DF64, OSB_FP32


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


def _bc(osb, sym):
    return tuple(osb.OSB_BC_SYMMETRIC if s else osb.OSB_BC_PERIODIC for s in sym)


def _state(nx, ny, nz, seed):
    return conserved(*inputs.smooth_primitive_state(nx, ny, nz, seed), gamma=1.4)


def _errs(Q, ref):
    """Relative L2 per field; momentum components against the momentum norm."""
    mnorm = np.linalg.norm(ref[1:4].ravel())
    return [np.linalg.norm((Q[m] - ref[m]).ravel()) / (mnorm if 1 <= m <= 3 else np.linalg.norm(ref[m].ravel()))
            for m in range(5)]


SYMS = [(True, True, True), (True, False, False), (False, True, False), (False, False, True), (False, True, True)]


@pytest.mark.parametrize("sym", SYMS)
@pytest.mark.parametrize("precision", [0, 2, 1])
def test_residual_and_steps_match_oracle(osb, sym, precision):
    nx, ny, nz = 20, 12, 10
    Q = _state(nx, ny, nz, 21)
    for order, visc in ((4, 0), (8, 0), (4, 1)):
        case = orc.Case(nx, ny, nz, order=order, visc_form=visc, Re=200.0, dt=1e-3)
        g = osb.Grid(osb.Config(nx, ny, nz, order=order, precision=precision, visc_form=visc, Re=200.0, dt=1e-3,
                                bc=_bc(osb, sym)))
        g.set_state(Q)
        R = g.residual().cpu().numpy()
        Ro = orc.sym_residual(case, Q, sym)
        g.step(3)
        S = g.get_state()
        So = orc.sym_rk3_step(case, Q, 3, sym)
        tol = TOL[precision]
        if precision != 1:
            scale = np.abs(Ro).max()
            assert np.abs(R - Ro).max() <= tol * scale, (order, visc)
        assert max(_errs(S, So)) < tol, (order, visc, _errs(S, So))


@pytest.mark.parametrize("order", [2, 6, 10, 12])
def test_every_order_fp64(osb, order):
    sym = (True, True, False)
    nx, ny, nz = 14, 16, 8
    Q = _state(nx, ny, nz, order)
    case = orc.Case(nx, ny, nz, order=order, Re=300.0, dt=5e-4)
    g = osb.Grid(osb.Config(nx, ny, nz, order=order, Re=300.0, dt=5e-4, bc=_bc(osb, sym)))
    g.set_state(Q)
    g.step(2)
    assert max(rel_l2_fields(g.get_state(), orc.sym_rk3_step(case, Q, 2, sym)).values()) < 1e-12


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 1), (3, 1, 2), (5, 2, 4)])
@pytest.mark.parametrize("precision", [0, 2, 1])
def test_extents_below_the_stencil_radius(osb, dims, precision):
    """Order 8 (radius 4) on axes of 1 to 5 points: neighbours mirror more
    than once before they land on a grid point."""
    nx, ny, nz = dims
    sym = (True, True, True)
    Q = _state(nx, ny, nz, 3 + nx)
    case = orc.Case(nx, ny, nz, order=8, Re=200.0, dt=1e-3)
    g = osb.Grid(osb.Config(nx, ny, nz, order=8, precision=precision, Re=200.0, dt=1e-3, bc=_bc(osb, sym)))
    g.set_state(Q)
    g.step(2)
    assert max(_errs(g.get_state(), orc.sym_rk3_step(case, Q, 2, sym))) < TOL[precision]


def test_tgv_octant_init_and_run_match_the_full_box(osb):
    """The vortex on [0, pi]^3 with symmetry planes against the GPU's periodic
    run of the whole box on the half-cell-shifted grid, restricted."""
    import torch
    n, steps = 16, 5
    sym = (True, True, True)
    case = orc.Case(n, n, n, order=4)
    g = osb.Grid(osb.Config(n, n, n, order=4, bc=_bc(osb, sym)))
    g.init_taylor_green()
    Q0 = g.get_state()
    assert rel_l2(Q0, orc.tgv_state(case, sym)) < 4e-15
    full0 = orc.sym_extend(Q0, sym)
    gf = osb.Grid(osb.Config(2 * n, 2 * n, 2 * n, order=4))
    gf.set_state(full0)
    g.step(steps)
    gf.step(steps)
    Qs, Qf = g.get_state(), orc.sym_restrict(gf.get_state(), case)
    assert max(rel_l2_fields(Qs, Qf).values()) < 1e-13
    assert max(rel_l2_fields(Qs, orc.sym_rk3_step(case, Q0, steps, sym)).values()) < 1e-12
    # diagnostics: means over the octant equal the full box's for the even
    # integrands
    d, df = g.diagnostics(), gf.diagnostics()
    for k in ("ke", "enstrophy"):
        assert abs(d[k] - df[k]) <= 1e-13 * abs(df[k])
    assert abs(d["total"][0] - df["total"][0]) <= 1e-14 * df["total"][0]
    assert abs(d["max_cfl"] - df["max_cfl"]) <= 1e-13 * df["max_cfl"]
    del gf
    torch.cuda.empty_cache()


def test_diagnostics_match_oracle(osb):
    sym = (True, False, True)
    nx, ny, nz = 12, 10, 8
    rho, u0, u1, u2, p = inputs.smooth_primitive_state(nx, ny, nz, seed=4)
    Q = conserved(rho, u0 + 0.3, u1, u2 - 0.2, p, gamma=1.4)
    case = orc.Case(nx, ny, nz, order=6, dt=2e-3)
    g = osb.Grid(osb.Config(nx, ny, nz, order=6, dt=2e-3, bc=_bc(osb, sym)))
    g.set_state(Q)
    d = g.diagnostics()
    do = orc.sym_diagnostics(case, Q, sym)
    assert abs(d["ke"] - do["ke"]) <= 1e-13 * do["ke"]
    assert abs(d["enstrophy"] - do["enstrophy"]) <= 1e-12 * do["enstrophy"]
    assert abs(d["max_cfl"] - do["max_cfl"]) <= 1e-13 * do["max_cfl"]
    keys = ("rho", "rhou0", "rhou1", "rhou2", "rhoE")
    for m, k in enumerate(keys):
        assert abs(d["total"][m] - do[k]) <= 1e-13 * max(abs(do[k]), 1e-3), k


@pytest.mark.parametrize("precision", [0, 1])
def test_euler_step(osb, precision):
    sym = (False, True, True)
    nx, ny, nz = 16, 12, 10
    Q = _state(nx, ny, nz, 8)
    case = orc.Case(nx, ny, nz, order=4, Re=200.0, dt=5e-4)
    g = osb.Grid(osb.Config(nx, ny, nz, order=4, precision=precision, Re=200.0, dt=5e-4, bc=_bc(osb, sym)))
    g.set_state(Q)
    g.euler_step(3)
    assert max(_errs(g.get_state(), orc.sym_euler_step(case, Q, 3, sym))) < TOL[precision]


def test_mass_and_energy_conserved(osb):
    sym = (True, True, True)
    n = 24
    g = osb.Grid(osb.Config(n, n, n, order=8, Re=100.0, dt=2e-3, bc=_bc(osb, sym)))
    rho, u0, u1, u2, p = inputs.smooth_primitive_state(n, n, n, seed=17)
    g.set_state(conserved(rho, u0 + 0.2, u1, u2, p))
    t0 = g.diagnostics()["total"]
    g.step(20)
    t1 = g.diagnostics()["total"]
    assert abs(t1[0] - t0[0]) <= 1e-13 * t0[0]
    assert abs(t1[4] - t0[4]) <= 1e-13 * t0[4]


def test_back_to_periodic_and_refusals(osb):
    import torch
    n = 16
    Q = _state(n, n, n, 5)
    g = osb.Grid(osb.Config(n, n, n, order=4, bc=_bc(osb, (True, True, True))))
    L = osb.load()
    # switch back: identical to a periodic grid
    assert L.osb_set_boundaries(g.handle, 0, 0, 0) == 0
    g.set_state(Q)
    g.step(2)
    gp = osb.Grid(osb.Config(n, n, n, order=4))
    gp.set_state(Q)
    gp.step(2)
    assert np.array_equal(g.get_state(), gp.get_state())
    # invalid kinds
    assert L.osb_set_boundaries(g.handle, 2, 0, 0) == 1
    assert L.osb_set_boundaries(g.handle, 0, -1, 0) == 1
    # ensembles and closures take periodic grids only
    assert L.osb_set_boundaries(g.handle, 0, 1, 0) == 0
    with pytest.raises(osb.OsbError) as e:
        osb.batch_step([g, gp], 1)
    assert e.value.status == 2
    from paper_1609_01277_gb300 import closure as clm
    c = clm.Closure(n, n, n, seed=1)
    assert L.osb_grid_set_closure(g.handle, c.handle) == 2
    assert L.osb_grid_set_closure(gp.handle, c.handle) == 0
    assert L.osb_set_boundaries(gp.handle, 1, 0, 0) == 2
    assert L.osb_grid_set_closure(gp.handle, None) == 0
    del c
    torch.cuda.synchronize()

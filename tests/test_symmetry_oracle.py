"""Pins of the oracle's symmetry boundaries (Section 2.6, "Boundary conditions").

The oracle runs a grid with symmetry planes as the periodic scheme on the
mirror-extended grid.  These tests pin that construction to what the paper
and the geometry fix:

* the extension carries exactly the halo values the paper's rule prescribes
  (scalars mirrored, the normal vector component mirrored with a sign change,
  at both ends of the axis, for halos as wide as the stencil and wider);
* a stencil applied through halos built one value at a time by that rule
  equals the stencil on the extended field (brute force on a tiny grid);
* the Taylor-Green vortex has mirror planes at 0 and pi: the extension of
  its state on [0, pi] is the vortex itself on the half-cell-shifted full box
  (evaluated independently), and the symmetric run equals the periodic run of
  that full box restricted to the first octant -- which fails for a wrong
  parity, a wrong mirror index or a wrong spacing;
* mass and energy cannot cross a symmetry plane: their totals are conserved
  on the symmetric grid, while the normal momentum is not (the wall pressure
  acts on it).
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs
from tests.helpers import conserved

SYMS = [(True, False, False), (False, True, False), (False, False, True), (True, True, True), (False, True, True)]


def _random_state(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((5, nz, ny, nx))


@pytest.mark.parametrize("sym", SYMS)
def test_extension_holds_the_paper_halo_rule(sym):
    nx, ny, nz = 5, 4, 3
    Q = _random_state(nx, ny, nz, 11)
    Qe = orc.sym_extend(Q, sym)
    n = (nx, ny, nz)
    for a in range(3):
        arr = 3 - a
        N = n[a]
        if not sym[a]:
            assert Qe.shape[arr] == N
            continue
        assert Qe.shape[arr] == 2 * N
        for m in range(5):
            sign = -1.0 if m == 1 + a else 1.0  # the momentum component normal to the plane
            for k in range(N):
                # after the last point: phi(x_{N+k}) = +-phi(x_{N-1-k})
                hi = np.take(Qe[m], N + k, axis=arr - 1)
                assert np.array_equal(hi, sign * np.take(Qe[m], N - 1 - k, axis=arr - 1))
                # before the first point (periodic image -1-k of the 2N axis):
                # phi(x_{-1-k}) = +-phi(x_k)
                lo = np.take(Qe[m], 2 * N - 1 - k, axis=arr - 1)
                assert np.array_equal(lo, sign * np.take(Qe[m], k, axis=arr - 1))


@pytest.mark.parametrize("order", [2, 4, 8])
def test_stencil_through_rule_built_halos_brute_force(order):
    """A first and a second derivative along a symmetric x axis, with halos of
    width r filled point by point by the paper's rule (multiple reflections
    where r exceeds N), against the periodic oracle stencil on the extension."""
    r = order // 2
    c, d = orc.fd_coeffs(order)
    for N in (1, 2, 3, 7):
        case = orc.Case(N, 1, 1, order=order)
        h = np.pi / N
        f = np.random.default_rng(N).standard_normal(N)
        for sign in (1.0, -1.0):  # an even and an odd field
            def val(j):
                # the rule applied until j is inside [0, N)
                s = 1.0
                while not 0 <= j < N:
                    if j >= N:
                        j = 2 * N - 1 - j
                    else:
                        j = -1 - j
                    s *= sign
                return s * f[j]
            bf1 = np.array([sum(c[k] * (val(i + k) - val(i - k)) for k in range(1, r + 1)) / h for i in range(N)])
            bf2 = np.array([(d[0] * val(i) + sum(d[k] * (val(i + k) + val(i - k)) for k in range(1, r + 1))) / h**2
                            for i in range(N)])
            fe = np.concatenate([f, sign * f[::-1]]).reshape(1, 1, 2 * N)
            ce = orc.sym_case(case, (True, False, False))
            o1 = orc.d1(ce, 0, fe).ravel()[:N]
            o2 = orc.d2(ce, 0, fe).ravel()[:N]
            assert np.allclose(o1, bf1, rtol=0, atol=1e-12 * max(1.0, np.abs(bf1).max()))
            assert np.allclose(o2, bf2, rtol=0, atol=1e-12 * max(1.0, np.abs(bf2).max()))


def _shifted(n):
    """Coordinates of a periodic [0, 2 pi) axis shifted by half a cell."""
    return (np.arange(n) + 0.5) * (2 * np.pi / n)


def test_tgv_state_matches_the_periodic_init():
    case = orc.Case(10, 8, 6)
    noise = inputs.gaussian_noise(10, 8, 6, 3)
    assert np.abs(orc.tgv_state(case, noise=noise, amp=1e-3) - orc.tgv_init(case, noise, 1e-3)).max() < 1e-12


@pytest.mark.parametrize("sym", SYMS)
def test_tgv_octant_is_the_full_vortex(sym):
    case = orc.Case(8, 6, 4, order=4, Re=400.0)
    Q = orc.tgv_state(case, sym)
    ce = orc.sym_case(case, sym)
    xs = [_shifted(n) if s else orc.axis_coords(n, False) for n, s in zip((ce.nx, ce.ny, ce.nz), sym)]
    full = orc.tgv_at(ce, *xs)
    assert np.abs(orc.sym_extend(Q, sym) - full).max() < 1e-12
    # residual and three RK3 steps of the symmetric grid vs the full box
    scale = np.abs(orc.residual(ce, full)).max()
    assert np.abs(orc.sym_residual(case, Q, sym) - orc.sym_restrict(orc.residual(ce, full), case)).max() < 1e-12 * scale
    Qs = orc.sym_rk3_step(case, Q, 3, sym)
    Qf = orc.sym_restrict(orc.rk3_step(ce, full, 3), case)
    assert np.abs(Qs - Qf).max() < 1e-12 * np.abs(Qf).max()


@pytest.mark.parametrize("visc_form", [0, 1])
def test_mass_and_energy_do_not_cross_symmetry_planes(visc_form):
    nx, ny, nz = 10, 8, 6
    Q = conserved(*inputs.smooth_primitive_state(nx, ny, nz, seed=5), gamma=1.4)
    case = orc.Case(nx, ny, nz, order=4, Re=100.0, dt=2e-3, visc_form=visc_form)
    sym = (True, True, True)
    Q1 = orc.sym_rk3_step(case, Q, 5, sym)
    # viscous work form B conserves the energy only to truncation error, on
    # periodic grids as well (Section 3.3 energy equation, product-rule form)
    for m in ((0, 4) if visc_form == 0 else (0,)):
        assert abs(Q1[m].sum() - Q[m].sum()) < 1e-12 * abs(Q[m].sum())
    # the wall pressure changes the normal momentum: a real flux, not roundoff
    assert abs(Q1[1].sum() - Q[1].sum()) > 1e-6 * np.abs(Q[1]).sum()


def test_symmetric_diagnostics_are_means_over_the_grid():
    case = orc.Case(8, 8, 8, order=4)
    sym = (True, True, True)
    Q = orc.tgv_state(case, sym)
    d = orc.sym_diagnostics(case, Q, sym)
    full = orc.diagnostics(orc.sym_case(case, sym), orc.sym_extend(Q, sym))
    for k in ("ke", "enstrophy", "rho", "rhoE", "max_cfl"):
        assert abs(d[k] - full[k]) <= 1e-13 * abs(full[k])
    # Taylor-Green kinetic energy at t = 0: <rho u^2/2> -> 1/8 as M -> 0
    assert abs(d["ke"] - 0.125) < 5e-3
    # a general state: the normal momentum's mean over the grid is its own,
    # the extension's is zero (odd under the mirror)
    rho, u0, u1, u2, p = inputs.smooth_primitive_state(8, 8, 8, seed=9)
    Q = conserved(rho, u0 + 0.3, u1, u2, p, gamma=1.4)
    d = orc.sym_diagnostics(case, Q, sym)
    full = orc.diagnostics(orc.sym_case(case, sym), orc.sym_extend(Q, sym))
    assert d["rhou0"] == Q[1].mean() and abs(d["rhou0"]) > 1e-3 and abs(full["rhou0"]) < 1e-14


@pytest.mark.parametrize("wrong", ["normal_momentum_even", "tangential_momentum_odd", "energy_odd"])
def test_planted_parity_mistakes_are_caught(monkeypatch, wrong):
    """A wrong parity in the extension makes the octant differ from the full
    vortex (the pin above), or breaks conservation."""
    bad = orc.SYM_PARITY.copy()
    if wrong == "normal_momentum_even":
        bad[1, 0] = 1.0
    elif wrong == "tangential_momentum_odd":
        bad[2, 0] = -1.0
    else:
        bad[4, 0] = -1.0
    monkeypatch.setattr(orc, "SYM_PARITY", bad)
    sym = (True, False, False)
    case = orc.Case(8, 6, 4, order=4, Re=400.0)
    ce = orc.sym_case(case, sym)
    full = orc.tgv_at(ce, _shifted(ce.nx), orc.axis_coords(ce.ny, False), orc.axis_coords(ce.nz, False))
    Q = orc.tgv_state(case, sym)
    assert np.abs(orc.sym_extend(Q, sym) - full).max() > 1e-3

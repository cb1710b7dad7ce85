"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test targets a class of mistake: a wrong weight, a wrong sign or axis in
a stencil, a dropped or mis-scaled term in the residual, a wrong RK
coefficient, a wrong initial state, a broken periodic wrap.
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs
from tests import bruteforce as bf
from tests.helpers import conserved, rel_l2

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Stencil weights (Section 2.4: arbitrary even order central differences)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
def test_fd_weights_match_taylor_matching(order):
    r = order // 2
    c, d = orc.fd_coeffs(order)
    cw = bf.first_derivative_weights(r)
    d0, dw = bf.second_derivative_weights(r)
    for k in range(1, r + 1):
        assert c[k] == float(cw[k - 1])          # correctly rounded rational
        assert d[k] == pytest.approx(float(dw[k - 1]), rel=2e-16, abs=0)
    assert d[0] == pytest.approx(float(d0), rel=4e-16)


def test_second_order_weight_printed_in_paper():
    g = _golden("paper_values.json")
    c, _ = orc.fd_coeffs(2)
    assert c[1] == g["second_order_first_derivative_weight_rc0"]["value"]


def test_fd_weights_known_rationals():
    # order 8 weights, as exact rationals
    c, d = orc.fd_coeffs(8)
    assert [Fraction(v).limit_denominator(10000) for v in c[1:]] == \
        [Fraction(4, 5), Fraction(-1, 5), Fraction(4, 105), Fraction(-1, 280)]
    assert Fraction(d[0]).limit_denominator(10000) == Fraction(-205, 72)


@pytest.mark.parametrize("order", [2, 4, 8, 12])
def test_polynomial_exactness_of_weights(order):
    """D is exact for degree <= 2r, D2 for degree <= 2r+1 (interior, unit h)."""
    r = order // 2
    c, d = orc.fd_coeffs(order)
    for deg in range(0, 2 * r + 1):
        # derivative at x=0 of x^deg
        approx = sum(c[k] * (k ** deg - (-k) ** deg) for k in range(1, r + 1))
        exact = 1.0 if deg == 1 else 0.0
        assert approx == pytest.approx(exact, abs=1e-9 * max(1, r ** deg))
    for deg in range(0, 2 * r + 2):
        approx = d[0] * (1.0 if deg == 0 else 0.0) + sum(
            d[k] * (k ** deg + (-k) ** deg) for k in range(1, r + 1))
        exact = 2.0 if deg == 2 else 0.0
        assert approx == pytest.approx(exact, abs=1e-9 * max(1, r ** deg))


# --------------------------------------------------------------------------
# Stencil application on the periodic grid: modified wavenumber
# --------------------------------------------------------------------------
def _kappa1(order, k, h):
    c, _ = orc.fd_coeffs(order)
    return sum(2 * c[m] * math.sin(m * k * h) for m in range(1, order // 2 + 1)) / h


def _kappa2(order, k, h):
    _, d = orc.fd_coeffs(order)
    return -(d[0] + sum(2 * d[m] * math.cos(m * k * h) for m in range(1, order // 2 + 1))) / h ** 2


@pytest.mark.parametrize("order,n", [(2, 8), (4, 8), (8, 8), (8, 6), (12, 5), (4, 13)])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_modified_wavenumber(order, n, axis):
    """D sin(kx) = kappa1(k) cos(kx) and D2 cos(kx) = -kappa2(k) cos(kx)
    exactly (to roundoff) on the periodic grid, including wrap-around."""
    dims = [n + 1, n + 2, n + 3]
    dims[axis] = n
    case = orc.Case(*dims, order=order)
    h = 2 * math.pi / n
    k = 2 if n > 4 else 1
    coord = 2 * math.pi * np.arange(n) / n
    shape = [1, 1, 1]
    shape[2 - axis] = n
    s = np.broadcast_to(np.sin(k * coord).reshape(shape), case.shape)
    co = np.broadcast_to(np.cos(k * coord).reshape(shape), case.shape)
    out1 = orc.d1(case, axis, s)
    out2 = orc.d2(case, axis, co)
    assert np.allclose(out1, _kappa1(order, k, h) * co, rtol=0, atol=1e-13)
    assert np.allclose(out2, -_kappa2(order, k, h) * co, rtol=0, atol=1e-12)
    # orthogonal axes see a constant: derivative zero
    for other in range(3):
        if other != axis:
            assert np.abs(orc.d1(case, other, s)).max() < 1e-13


# --------------------------------------------------------------------------
# Full residual against the continuous equations (manufactured solution)
# --------------------------------------------------------------------------
_MMS = dict(Re=20.0, Mach=0.5, gamma=1.4, Pr=0.71)


def _mms_exact():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    Re, M, g, Pr = (sp.Rational(str(v)) for v in (_MMS["Re"], _MMS["Mach"], _MMS["gamma"], _MMS["Pr"]))
    rho = 1 + sp.Rational(1, 5) * sp.sin(x) * sp.cos(2 * y) + sp.Rational(1, 10) * sp.cos(z)
    # div u depends on x, y and z, so every d_i (div u) term is exercised
    u = [sp.sin(x) * sp.cos(y) * sp.cos(z) + sp.Rational(3, 10) * sp.sin(y + z)
         + sp.Rational(1, 10) * sp.cos(x + 2 * y),
         -sp.cos(x) * sp.sin(y) * sp.cos(z) + sp.Rational(1, 5) * sp.cos(x - z)
         + sp.Rational(3, 20) * sp.sin(2 * y + z),
         sp.Rational(3, 10) * sp.sin(x) * sp.sin(2 * z) + sp.Rational(1, 10) * sp.cos(y)]
    p = 1 / (g * M ** 2) + sp.Rational(1, 2) * sp.cos(x + y) * sp.sin(z)
    T = g * M ** 2 * p / rho
    rhoE = p / (g - 1) + rho * sum(ui ** 2 for ui in u) / 2
    div = sum(sp.diff(u[k], X[k]) for k in range(3))
    tau = [[(sp.diff(u[i], X[j]) + sp.diff(u[j], X[i]) - (sp.Rational(2, 3) * div if i == j else 0)) / Re
            for j in range(3)] for i in range(3)]
    kappa = 1 / ((g - 1) * M ** 2 * Pr * Re)
    q = [kappa * sp.diff(T, X[j]) for j in range(3)]
    # conservative form exactly as printed (mass, momentum, energy equations)
    R = [-sum(sp.diff(rho * u[j], X[j]) for j in range(3))]
    for i in range(3):
        R.append(-sum(sp.diff(rho * u[i] * u[j] + (p if i == j else 0) - tau[i][j], X[j]) for j in range(3)))
    R.append(-sum(sp.diff(rhoE * u[j] + u[j] * p - q[j] - sum(u[i] * tau[i][j] for i in range(3)), X[j])
                  for j in range(3)))
    prim = [rho, u[0], u[1], u[2], p]
    fprim = sp.lambdify(X, prim, "numpy")
    fR = [sp.lambdify(X, r, "numpy") for r in R]
    return fprim, fR


@pytest.fixture(scope="module")
def mms():
    return _mms_exact()


def _mms_error(mms, n, order, visc_form):
    """Per-field max error of the discrete residual, relative to max |R_exact|."""
    fprim, fR = mms
    c = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    prim = [np.broadcast_to(np.asarray(v, dtype=float), X.shape) for v in fprim(X, Y, Z)]
    Q = conserved(*prim, gamma=_MMS["gamma"])
    case = orc.Case(n, n, n, order=order, visc_form=visc_form, **_MMS)
    Rh = orc.residual(case, Q)
    err = []
    for m in range(5):
        Re = np.broadcast_to(np.asarray(fR[m](X, Y, Z), dtype=float), X.shape)
        err.append(np.abs(Rh[m] - Re).max() / np.abs(Re).max())
    return np.array(err)


@pytest.mark.parametrize("order,n0", [(2, 16), (4, 24), (6, 32), (8, 32)])
@pytest.mark.parametrize("visc_form", [0, 1])
def test_residual_converges_to_continuous_equations(mms, order, n0, visc_form):
    """||R_h - R_exact|| falls like h^order in every equation (the MMS idea of
    Section 3.2 applied to the full Navier-Stokes residual of Section 3.3,
    with Re = 20 so that the viscous and heat-flux terms are not negligible).
    A dropped, mis-signed or mis-scaled term leaves an O(1) plateau and a
    slope near zero."""
    e1 = _mms_error(mms, n0, order, visc_form)
    e2 = _mms_error(mms, 2 * n0, order, visc_form)
    slope = np.log2(e1 / e2)
    assert np.all(slope > order - 1.0), (e1, e2, slope)
    assert np.all(slope < order + 1.0), (e1, e2, slope)


# --------------------------------------------------------------------------
# Invariants of the discrete scheme
# --------------------------------------------------------------------------
def test_uniform_state_has_zero_residual():
    case = orc.Case(9, 8, 7, order=8)
    one = np.ones(case.shape)
    Q = conserved(1.3 * one, 0.4 * one, -0.2 * one, 0.7 * one, 50.0 * one)
    R = orc.residual(case, Q)
    assert np.abs(R).max() < 1e-10


@pytest.mark.parametrize("order", [2, 4, 8])
def test_residual_sums_to_zero_form_a(order):
    """Form A: every term is a central difference of something, or a skew
    pair a D b + b D a, so each conserved total has zero rate to roundoff."""
    case = orc.Case(12, 10, 14, order=order, visc_form=0, Re=50.0)
    Q = conserved(*inputs.smooth_primitive_state(12, 10, 14, seed=3))
    R = orc.residual(case, Q)
    scale = np.abs(R).max(axis=(1, 2, 3))
    for m in range(5):
        assert abs(R[m].sum()) / R[m].size < 1e-13 * max(scale[m], 1.0), m


def test_form_b_energy_rate_is_truncation_level():
    """Form B (product rule on u_i tau_ij) conserves energy only up to the
    truncation error: nonzero, and falling with h."""
    rates = []
    for n in (12, 24):
        case = orc.Case(n, n, n, order=4, visc_form=1, Re=20.0)
        Q = conserved(*inputs.smooth_primitive_state(n, n, n, seed=5))
        R = orc.residual(case, Q)
        rates.append(abs(R[4].mean()))
    assert rates[0] > 1e-10
    assert rates[1] < rates[0] / 4


def test_conservation_over_steps():
    case = orc.Case(16, 16, 16, order=4, dt=2e-3)
    Q = conserved(*inputs.smooth_primitive_state(16, 16, 16, seed=11), gamma=case.gamma)
    tot0 = Q.sum(axis=(1, 2, 3))
    Q = orc.rk3_step(case, Q, 10)
    tot1 = Q.sum(axis=(1, 2, 3))
    absq = np.abs(Q).sum(axis=(1, 2, 3))
    assert np.all(np.abs(tot1 - tot0) <= 1e-14 * 10 * 3 * absq + 1e-300)


def test_tgv_reflection_symmetry_is_preserved():
    """TGV is symmetric under x -> -x (u0 odd, the rest even); a central
    scheme keeps this to roundoff for any number of steps."""
    n = 16
    case = orc.Case(n, n, n, order=4)
    Q = orc.rk3_step(case, orc.tgv_init(case), 5)
    ref = np.roll(Q[:, :, :, ::-1], 1, axis=3)   # index i -> (N - i) mod N
    sign = np.array([1, -1, 1, 1, 1]).reshape(5, 1, 1, 1)
    assert np.abs(Q - sign * ref).max() < 1e-12 * np.abs(Q).max()
    # y reflection: u1 odd
    ref = np.roll(Q[:, :, ::-1, :], 1, axis=2)
    sign = np.array([1, 1, -1, 1, 1]).reshape(5, 1, 1, 1)
    assert np.abs(Q - sign * ref).max() < 1e-12 * np.abs(Q).max()


# --------------------------------------------------------------------------
# Time integration (low-storage RK3)
# --------------------------------------------------------------------------
def test_rk3_order_conditions_exact():
    a, b = orc.rk3_coeffs()
    A = [Fraction(v).limit_denominator(100) for v in a]
    B = [Fraction(v).limit_denominator(100) for v in b]
    assert [float(v) for v in A] == list(a) and [float(v) for v in B] == list(b)
    # Butcher form of the 2-register scheme
    c2 = A[0]
    a31, a32 = B[0], A[1]
    c3 = a31 + a32
    assert sum(B) == 1
    assert B[1] * c2 + B[2] * c3 == Fraction(1, 2)
    assert B[1] * c2 ** 2 + B[2] * c3 ** 2 == Fraction(1, 3)
    assert B[2] * a32 * c2 == Fraction(1, 6)
    assert A[2] == B[2]   # last stage: q_3 = U_3


def test_rk3_linear_stability_polynomial():
    lam = np.array([-1.0, -3.0, 0.5, -0.1])
    dt, nsteps = 0.1, 7
    y = orc.rk3_linear(lam, np.ones(4), nsteps, dt)
    z = lam * dt
    P = 1 + z + z ** 2 / 2 + z ** 3 / 6
    assert np.allclose(y, P ** nsteps, rtol=1e-14, atol=0)


def test_rk3_temporal_order_is_three():
    lam = np.array([-2.0])
    errs = []
    for nsteps in (20, 40, 80):
        y = orc.rk3_linear(lam, np.ones(1), nsteps, 1.0 / nsteps)
        errs.append(abs(y[0] - math.exp(-2.0)))
    s1 = math.log2(errs[0] / errs[1])
    s2 = math.log2(errs[1] / errs[2])
    assert 2.9 < s1 < 3.1 and 2.9 < s2 < 3.1


def test_forward_euler_linear_closed_form_and_first_order():
    """Forward Euler (Section 2.4): y_n = (1 + lambda dt)^n y_0 exactly, and the
    error against exp(lambda t) halves with dt."""
    lam = np.array([-1.0, -3.0, 0.5, -0.1])
    dt, nsteps = 0.1, 7
    y = orc.euler_linear(lam, np.ones(4), nsteps, dt)
    assert np.allclose(y, (1 + lam * dt) ** nsteps, rtol=1e-14, atol=0)
    errs = []
    for n in (40, 80, 160):
        errs.append(abs(orc.euler_linear(np.array([-2.0]), np.ones(1), n, 1.0 / n)[0] - math.exp(-2.0)))
    for e0, e1 in zip(errs, errs[1:]):
        assert 0.9 < math.log2(e0 / e1) < 1.1


def test_forward_euler_conserves_totals_and_is_one_stage_of_the_residual():
    """Each forward-Euler step adds dt R, whose totals vanish (form A), so the
    conserved totals stay put to roundoff; and a step from the uniform state
    leaves it unchanged (R = 0)."""
    case = orc.Case(16, 16, 16, order=4, dt=2e-3)
    Q = conserved(*inputs.smooth_primitive_state(16, 16, 16, seed=11), gamma=case.gamma)
    Q1 = orc.euler_step(case, Q, 5)
    for m in range(5):
        assert abs(Q1[m].sum() - Q[m].sum()) <= 1e-12 * np.abs(Q[m]).sum()
    one = np.ones(case.shape)
    U = conserved(1.3 * one, 0.4 * one, -0.2 * one, 0.7 * one, 50.0 * one)
    assert np.allclose(orc.euler_step(case, U, 3), U, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# Taylor-Green initial state (Section 3.3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,order", [(8, 4), (16, 2), (32, 4), (24, 8)])
def test_tgv_initial_kinetic_energy_and_enstrophy(n, order):
    """E_k(0) = 1/8 exactly on any grid with N not in {1,2,4}; the discrete
    enstrophy is kappa1^2 (3/8 - 5 gamma M^2 / 128) with kappa1 the modified
    wavenumber of mode 1 (closed forms derived from the initial state)."""
    case = orc.Case(n, n, n, order=order)
    Q = orc.tgv_init(case)
    dg = orc.diagnostics(case, Q)
    k1 = _kappa1(order, 1, 2 * math.pi / n)
    gM2 = case.gamma * case.Mach ** 2
    assert dg["ke"] == pytest.approx(0.125, rel=1e-14)
    assert dg["enstrophy"] == pytest.approx(k1 ** 2 * (3 / 8 - 5 * gM2 / 128), rel=1e-13)
    assert dg["rho"] == pytest.approx(1.0, rel=1e-14)
    for m in ("rhou0", "rhou1", "rhou2"):
        assert abs(dg[m]) < 1e-15
    assert dg["rhoE"] == pytest.approx(1 / (gM2 * (case.gamma - 1)) + 0.125, rel=1e-13)
    assert dg["nonfinite"] == 0


def test_tgv_golden_enstrophy_values():
    g = _golden("tgv_enstrophy0.json")
    for row in g["cases"]:
        case = orc.Case(row["n"], row["n"], row["n"], order=row["order"])
        dg = orc.diagnostics(case, orc.tgv_init(case))
        assert dg["enstrophy"] == pytest.approx(row["enstrophy0"], rel=1e-13)


def test_tgv_noise_perturbs_velocity_at_fixed_rho_and_p():
    n = 8
    case = orc.Case(n, n, n)
    noise = inputs.gaussian_noise(n, n, n, seed=1234)
    Q0 = orc.tgv_init(case)
    Q1 = orc.tgv_init(case, noise, 1e-4)
    assert np.array_equal(Q0[0], Q1[0])
    u0, p0, _ = orc.primitives(case, Q0)
    u1, p1, _ = orc.primitives(case, Q1)
    assert np.allclose(u1 - u0, 1e-4 * noise, atol=1e-15)
    assert np.allclose(p1, p0, rtol=1e-13)


def test_diagnostics_cfl_and_nonfinite_closed_form():
    case = orc.Case(8, 10, 12, dt=1e-3)
    one = np.ones(case.shape)
    rho, U, p = 1.2, 0.7, 40.0
    Q = conserved(rho * one, U * one, 0 * one, 0 * one, p * one, gamma=case.gamma)
    c = math.sqrt(case.gamma * p / rho)
    h = [2 * math.pi / v for v in (8, 10, 12)]
    cfl = case.dt * ((U + c) / h[0] + c / h[1] + c / h[2])
    dg = orc.diagnostics(case, Q)
    assert dg["max_cfl"] == pytest.approx(cfl, rel=1e-14)
    assert dg["ke"] == pytest.approx(0.5 * rho * U * U, rel=1e-14)
    assert dg["enstrophy"] == 0.0
    Q[2, 3, 4, 5] = np.nan
    Q[4, 0, 0, 0] = np.inf
    assert orc.diagnostics(case, Q)["nonfinite"] == 2


# --------------------------------------------------------------------------
# Brute force at 50 digits on tiny grids
# --------------------------------------------------------------------------
@pytest.mark.parametrize("order,visc_form", [(4, 0), (8, 0), (4, 1)])
def test_residual_matches_50_digit_bruteforce(order, visc_form):
    n = 8
    case = orc.Case(n, n, n, order=order, visc_form=visc_form, Re=40.0)
    noise = inputs.gaussian_noise(n, n, n, seed=7)
    Q = orc.tgv_init(case, noise, 0.05)
    R = orc.residual(case, Q)
    box = bf.Box(n, n, n, order)
    Rd = bf.to_float(bf.residual(box, bf.from_numpy(Q), case.Re, case.Mach, case.gamma, case.Pr,
                                 visc_form)).reshape(R.shape)
    for m in range(5):
        assert rel_l2(R[m], Rd[m]) < 1e-13, m


def test_rk3_step_matches_50_digit_bruteforce():
    n = (8, 6, 5)
    case = orc.Case(*n, order=4, Re=100.0, dt=5e-3)
    Q0 = conserved(*inputs.smooth_primitive_state(*n, seed=21), gamma=case.gamma)
    Q = orc.rk3_step(case, Q0, 2)
    box = bf.Box(*n, 4)
    Qd = bf.to_float(bf.rk3(box, bf.from_numpy(Q0), 2, case.dt, case.Re, case.Mach, case.gamma,
                            case.Pr)).reshape(Q.shape)
    for m in range(5):
        assert rel_l2(Q[m], Qd[m]) < 1e-14, m

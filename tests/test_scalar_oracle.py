"""Pins of the oracle's scalar advection-diffusion solver (Section 3.1 wave
propagation, Section 3.2 manufactured solution) against closed forms and the
paper's printed result.

A single Fourier mode is an eigenvector of every periodic central stencil:
D e^{ix} = i k1(h) e^{ix} with the modified wavenumber
k1 = (2/h) sum_k c_k sin(kh), and L e^{ix} = -k2(h) e^{ix} with
k2 = -(1/h^2)(d_0 + 2 sum_k d_k cos(kh)).  For a linear problem every
3-stage third-order Runge-Kutta scheme multiplies such a mode by
P(z) = 1 + z + z^2/2 + z^3/6 per step.  These give the exact discrete
solutions the oracle must reproduce to rounding."""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _symbols(order: int, n: int):
    c, d = orc.fd_coeffs(order)
    h = 2 * math.pi / n
    r = order // 2
    k1 = 2.0 / h * sum(c[k] * math.sin(k * h) for k in range(1, r + 1))
    k2 = -(d[0] + 2.0 * sum(d[k] * math.cos(k * h) for k in range(1, r + 1))) / h ** 2
    return k1, k2


def _P(z):
    return 1 + z + z * z / 2 + z ** 3 / 6


def _wave_case():
    w = json.load(open(GOLDEN))["wave_test"]
    n = int(round(1.0 / w["dx"]))
    steps = int(round(w["t_end"] / w["dt"]))
    # the paper's line 0 <= x < 1 maps to [0, 2 pi): x' = 2 pi x, speed 2 pi c,
    # the same discrete system (c dt / dx is unchanged)
    return w, n, steps, 2 * math.pi * w["c"]


def test_wave_equals_closed_form_discrete_solution():
    w, n, steps, a = _wave_case()
    case = orc.Case(n, 1, 1, order=w["order"], dt=w["dt"])
    x = np.arange(n) * 2 * math.pi / n
    phi = orc.scalar_rk3(case, np.sin(x).reshape(1, 1, n), adv=(a, 0, 0), nsteps=steps).ravel()
    k1, _ = _symbols(w["order"], n)
    Pn = _P(-1j * a * k1 * w["dt"]) ** steps
    exact_discrete = Pn.real * np.sin(x) + Pn.imag * np.cos(x)
    assert np.max(np.abs(phi - exact_discrete)) < 1e-12


def test_wave_error_matches_paper_order_of_magnitude():
    """Section 3.1: eighth order, Courant 0.2, t = 1: error O(1e-10)."""
    w, n, steps, a = _wave_case()
    case = orc.Case(n, 1, 1, order=w["order"], dt=w["dt"])
    x = np.arange(n) * 2 * math.pi / n
    phi = orc.scalar_rk3(case, np.sin(x).reshape(1, 1, n), adv=(a, 0, 0), nsteps=steps).ravel()
    err = np.max(np.abs(phi - np.sin(x - a * w["t_end"])))
    mag = w["error_order_of_magnitude"]
    assert mag / 10 <= err <= mag * 10, err


# --------------------------------------------------------------------------
# Section 3.2: d phi/dt + d_j(phi u_j - k d_j phi) + S = 0 on [0, 2 pi)^2,
# u = (1, -0.5), k = 0.75, phi_m = sin x0 cos x1, phi(t = 0) = 0.
MMS = dict(u=(1.0, -0.5), k=0.75)


def mms_source(n: int) -> np.ndarray:
    """S such that phi_m is the exact steady solution of the continuous equation:
    S = -(u0 cos x0 cos x1 - u1 sin x0 sin x1 + 2 k sin x0 cos x1)."""
    u0, u1, k = MMS["u"][0], MMS["u"][1], MMS["k"]
    x = np.arange(n) * 2 * math.pi / n
    X0, X1 = np.meshgrid(x, x, indexing="xy")  # X0 varies along the last axis (x0 fastest)
    S = -(u0 * np.cos(X0) * np.cos(X1) - u1 * np.sin(X0) * np.sin(X1) + 2 * k * np.sin(X0) * np.cos(X1))
    return S.reshape(1, n, n)


def mms_discrete_steady(order: int, n: int) -> np.ndarray:
    """Exact steady state of the semi-discrete equation in the 4-mode space
    {s0 c1, c0 s1, c0 c1, s0 s1} (s0 = sin x0, c1 = cos x1, ...)."""
    u0, u1, k = MMS["u"][0], MMS["u"][1], MMS["k"]
    k1, k2 = _symbols(order, n)
    # D0: s0 -> k1 c0, c0 -> -k1 s0;  L0: s0 -> -k2 s0, c0 -> -k2 c0 (same along x1)
    # basis index: 0 s0c1, 1 c0s1, 2 c0c1, 3 s0s1
    M = np.zeros((4, 4))
    lap = -2 * k * k2
    for j in range(4):
        M[j, j] += lap
    # -u0 D0: s0c1 -> -u0 k1 c0c1 ; c0s1 -> +u0 k1 s0s1 ; c0c1 -> +u0 k1 s0c1 ; s0s1 -> -u0 k1 c0s1
    M[2, 0] += -u0 * k1
    M[3, 1] += u0 * k1
    M[0, 2] += u0 * k1
    M[1, 3] += -u0 * k1
    # -u1 D1: s0c1 -> +u1 k1 s0s1 ; c0s1 -> -u1 k1 c0c1 ; c0c1 -> +u1 k1 c0s1 ; s0s1 -> -u1 k1 s0c1
    M[3, 0] += u1 * k1
    M[2, 1] += -u1 * k1
    M[1, 2] += u1 * k1
    M[0, 3] += -u1 * k1
    s = np.array([-2 * k, 0.0, -u0, u1])  # S in the basis
    a = np.linalg.solve(M, s)
    x = np.arange(n) * 2 * math.pi / n
    X0, X1 = np.meshgrid(x, x, indexing="xy")
    phi = (a[0] * np.sin(X0) * np.cos(X1) + a[1] * np.cos(X0) * np.sin(X1) +
           a[2] * np.cos(X0) * np.cos(X1) + a[3] * np.sin(X0) * np.sin(X1))
    return phi.reshape(1, n, n)


def mms_run(order: int, n: int, t_end: float = 25.0, cfl: float = 0.025):
    """Oracle run from phi = 0 at the paper's Courant bound (dt = cfl h / max|u|)."""
    h = 2 * math.pi / n
    dt = cfl * h / max(abs(v) for v in MMS["u"])
    steps = int(math.ceil(t_end / dt))
    case = orc.Case(n, n, 1, order=order, dt=dt)
    return orc.scalar_rk3(case, np.zeros((1, n, n)), adv=(MMS["u"][0], MMS["u"][1], 0.0), k=MMS["k"],
                          S=mms_source(n), nsteps=steps)


def test_mms_source_makes_phi_m_steady_for_the_continuous_operator():
    """Closed-form check of S itself on a fine grid: the spectral derivative of
    phi_m (exact for a single mode) balances S."""
    n = 16
    x = np.arange(n) * 2 * math.pi / n
    X0, X1 = np.meshgrid(x, x, indexing="xy")
    u0, u1, k = MMS["u"][0], MMS["u"][1], MMS["k"]
    d0 = np.cos(X0) * np.cos(X1)
    d1 = -np.sin(X0) * np.sin(X1)
    lap = -2 * np.sin(X0) * np.cos(X1)
    rhs = -(u0 * d0 + u1 * d1) + k * lap - mms_source(n)[0]
    assert np.max(np.abs(rhs)) < 1e-14


@pytest.mark.parametrize("order,n", [(2, 8), (4, 16), (8, 16), (12, 32)])
def test_mms_oracle_reaches_the_discrete_steady_state(order, n):
    phi = mms_run(order, n)
    assert np.max(np.abs(phi - mms_discrete_steady(order, n))) < 1e-11


def test_mms_convergence_slopes_match_the_orders():
    """Section 3.2: the steady error |phi_h - phi_m| falls as h^order for
    orders 2..12 under dx = pi/2 .. pi/32; the twelfth order meets rounding at
    the finest grids (the anomaly the paper reports)."""
    ns = [4, 8, 16, 32, 64]
    for order in (2, 4, 6, 8, 10, 12):
        errs = []
        for n in ns:
            x = np.arange(n) * 2 * math.pi / n
            X0, X1 = np.meshgrid(x, x, indexing="xy")
            pm = np.sin(X0) * np.cos(X1)
            errs.append(np.sqrt(np.mean((mms_discrete_steady(order, n)[0] - pm) ** 2)))
        usable = [(n, e) for n, e in zip(ns, errs) if e > 1e-12 and n >= 8]
        slopes = [math.log(e0 / e1, 2) for (n0, e0), (n1, e1) in zip(usable, usable[1:])]
        assert slopes, order
        assert abs(slopes[-1] - order) < 0.35, (order, slopes)
    assert errs[-1] < 1e-13  # order 12 at dx = pi/32: at the rounding floor

"""Pins of the closure-network oracle (CPU only): the backward pass against
central finite differences of the forward pass in exact FP64, the adjoint
identity of the convolution, and the box filter's invariants."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import closure_oracle as co


def _problem(seed=0, n=(8, 4, 4)):
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = n
    theta = rng.standard_normal(co.param_count()) * 0.1
    Q = rng.standard_normal((5, nz, ny, nx))
    C = rng.standard_normal((5, nz, ny, nx))
    mean, std, out = rng.standard_normal(5) * 0.1, 1 + rng.random(5), 1 + rng.random(5)
    return theta, Q, C, mean, std, out


def test_param_count():
    assert co.param_count() == 32 * 5 * 27 + 32 + 32 * 32 * 27 + 32 + 5 * 32 * 27 + 5 == 36357


def test_conv_adjoint_identity():
    rng = np.random.Generator(np.random.PCG64(1))
    x = rng.standard_normal((3, 4, 5, 6))
    d = rng.standard_normal((2, 4, 5, 6))
    W = rng.standard_normal((2, 3, 27))
    assert np.sum(co.conv(x, W) * d) == pytest.approx(np.sum(x * co.conv_t(d, W)), rel=1e-12)
    # and the weight gradient is the derivative of <conv(x, W), d> in W
    assert np.sum(co.wgrad(d, x) * W) == pytest.approx(np.sum(co.conv(x, W) * d), rel=1e-12)


def test_conv_single_tap_is_a_shift():
    x = np.arange(4 * 4 * 8, dtype=float).reshape(1, 4, 4, 8)
    W = np.zeros((1, 1, 27))
    W[0, 0, 2 * 9 + 1 * 3 + 2] = 1.0      # dz=+1, dy=0, dx=+1
    y = co.conv(x, W)
    assert np.array_equal(y[0, 1, 2, 3], x[0, 2, 2, 4])
    assert np.array_equal(y[0, 3, 0, 7], x[0, 0, 0, 0])   # periodic wrap in x and z


def test_backward_matches_finite_differences_exact():
    theta, Q, C, mean, std, out = _problem()
    _, g = co.loss_grad(theta, Q, C, mean, std, out, mode="exact")
    rng = np.random.Generator(np.random.PCG64(2))
    idx = rng.choice(theta.size, size=40, replace=False)
    idx = np.concatenate([idx, [co.param_count() - 1, 32 * 5 * 27]])  # a b3 and a b1 entry
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (co.loss_grad(tp, Q, C, mean, std, out, "exact")[0] - co.loss_grad(tm, Q, C, mean, std, out, "exact")[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.140625])
    assert np.array_equal(co.bf16(x), [1.0, 1.0, 1.0 + 4 * 2 ** -8, -2.5, 3.140625])


def test_box_filter_invariants():
    rng = np.random.Generator(np.random.PCG64(3))
    Q = rng.standard_normal((5, 8, 8, 16))
    F = co.box_filter(Q, 4)
    assert F.shape == (5, 2, 2, 4)
    assert np.allclose(F.mean(axis=(1, 2, 3)), Q.mean(axis=(1, 2, 3)), rtol=0, atol=1e-15)
    assert np.allclose(co.box_filter(np.full((5, 4, 4, 4), 2.5), 2), 2.5)
    assert F[1, 0, 1, 2] == pytest.approx(Q[1, 0:4, 4:8, 8:12].mean(), rel=1e-14)


def test_adam_closed_form_first_step():
    """First bias-corrected Adam step moves every parameter by lr * sign(g)
    (up to eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = co.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 0.01, 1)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-4)


def test_dissipative_correction_never_feeds_kinetic_energy():
    """The clipped momentum correction satisfies u . C_m <= 0 at every point,
    leaves points with u . C_m <= 0 untouched and only removes the component
    along u (the perpendicular part is kept)."""
    rng = np.random.default_rng(4)
    shape = (8, 4, 4)
    theta = rng.standard_normal(co.param_count()) * 0.05
    Q = np.empty((5,) + shape)
    Q[0] = 1.0 + 0.1 * rng.random(shape)
    Q[1:4] = rng.standard_normal((3,) + shape)
    Q[4] = 50.0 + rng.random(shape)
    mean, std, out = np.zeros(5), np.ones(5), np.full(5, 0.3)
    C0 = co.correction(theta, Q, mean, std, out, mode="exact")
    C1 = co.correction(theta, Q, mean, std, out, mode="exact", dissipative=True)
    u = Q[1:4] / Q[0]
    d0, d1 = np.sum(u * C0[1:4], axis=0), np.sum(u * C1[1:4], axis=0)
    assert np.all(d1 <= 1e-12 * np.sum(np.abs(u * C0[1:4]), axis=0))
    keep = d0 <= 0
    assert np.array_equal(C1[:, keep], C0[:, keep])
    assert keep.sum() > 0 and (~keep).sum() > 0
    # the removed part is parallel to u
    diff = C0[1:4] - C1[1:4]
    cross = np.cross(diff, u, axis=0)
    assert np.max(np.abs(cross)) < 1e-12 * max(1.0, np.max(np.abs(diff)))
    assert np.array_equal(C1[[0, 4]], C0[[0, 4]])

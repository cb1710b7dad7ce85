"""The seeded input recipes: reproducible, with the stated distributions and
the time-step rule of the uneven ensemble."""
from __future__ import annotations

import numpy as np

from paper_1609_01277_gb300 import inputs


def test_noise_is_seeded_standard_normal():
    a = inputs.gaussian_noise(16, 12, 8, 1234)
    b = inputs.gaussian_noise(16, 12, 8, 1234)
    assert a.shape == (3, 8, 12, 16) and np.array_equal(a, b)
    assert not np.array_equal(a, inputs.gaussian_noise(16, 12, 8, 1235))
    assert abs(a.mean()) < 0.05 and abs(a.std() - 1.0) < 0.05


def test_ensemble_recipe_and_time_step_rule():
    e = inputs.ensemble_with_dt(64, 7)
    assert e == inputs.ensemble_with_dt(64, 7) and len(e) == 64
    assert {x["n"] for x in e} <= {32, 48, 64, 96, 128}
    assert all(100.0 <= x["Re"] <= 3200.0 and 0.05 <= x["Mach"] <= 0.3 for x in e)
    # acoustic Courant number dt (|u| + c)/h with |u| ~ 1, c = 1/M, h = 2 pi / N:
    # the same for every instance as for the 64^3, M = 0.1 case
    ref = 3.385e-3 * (1.0 + 1.0 / 0.1) * 64 / (2 * np.pi)
    for x in e:
        cfl = x["dt"] * (1.0 + 1.0 / x["Mach"]) * x["n"] / (2 * np.pi)
        assert abs(cfl - ref) < 1e-12 * ref


def test_smooth_state_is_physical():
    rho, u0, u1, u2, p = inputs.smooth_primitive_state(12, 10, 8, seed=3)
    assert rho.shape == (8, 10, 12) and rho.min() > 0 and p.min() > 0
    assert max(np.abs(u).max() for u in (u0, u1, u2)) < 3.0

"""Host-side helpers of the experiments driver: dissipation rate, curve
summaries and run comparisons, on synthetic series with known answers."""
from __future__ import annotations

import numpy as np

from paper_1609_01277_gb300 import experiments as ex


def _run(ke_fn, t_end=2.0, dt=0.01, every=10, precision="fp64"):
    n = int(round(t_end / dt))
    t_step = [i * dt for i in range(n + 1)]
    ke_step = [ke_fn(t) for t in t_step]
    t = t_step[::every]
    ke = ke_step[::every]
    return dict(n=8, order=4, precision=precision, steps=n, dt=dt, seconds=1.0, point_stages_per_s=1.0,
                t=t, ke=ke, enstrophy=[1.0 + x for x in t], max_cfl=[0.5] * len(t),
                t_step=t_step, ke_step=ke_step, enstrophy_step=[1.0 + x for x in t_step], every=every)


def test_dissipation_of_a_known_decay():
    t = np.linspace(0.0, 2.0, 201)
    ke = 0.125 * np.exp(-0.5 * t)
    eps = ex.dissipation(t, ke)
    # second-order central differences inside, one-sided at the ends
    assert np.max(np.abs(eps[1:-1] - 0.0625 * np.exp(-0.5 * t[1:-1]))) < 1e-5


def test_summarize_uses_every_step_for_fp64_and_the_reductions_for_fp32():
    c = _run(lambda t: 0.125 - 0.01 * t * t)      # eps = 0.02 t, peak at the end
    s = ex.summarize(c)
    assert abs(s["t_max_dissipation"] - 2.0) < 1e-12
    assert abs(s["max_dissipation"] - 0.04) < 1e-3
    c32 = dict(c, precision="fp32", ke_step=[k + (1e-6 if i % 2 else 0.0) for i, k in enumerate(c["ke_step"])])
    s32 = ex.summarize(c32)                        # the noisy per-step series is not differentiated
    assert abs(s32["max_dissipation"] - 0.04) < 1e-3


def test_compare_curves_reports_both_ke_errors():
    a = _run(lambda t: 0.125 - 0.01 * t)
    b = _run(lambda t: 0.125 - 0.01 * t + 1e-4 * np.sin(7.3 * t))
    r = ex.compare_curves(b, a)
    assert abs(r["ke_err_every_step"] - 1e-4 / 0.125) < 2e-5
    assert r["ke_err"] <= r["ke_err_every_step"] + 1e-15
    assert r["speedup"] == 1.0


def test_series_csv_rows_and_dissipation(tmp_path):
    """The CSV writer's columns on a series with a known decay rate."""
    dt, Re = 0.01, 1600.0
    t = np.arange(101) * dt
    ke = 0.125 * np.exp(-0.5 * t)
    ens = 0.2 + 0.1 * t
    path = tmp_path / "series.csv"
    ex.write_series_csv(str(path), ke, ens, dt, Re, step0=3)
    lines = path.read_text().splitlines()
    assert lines[0] == "step,t,ke,enstrophy,dissipation,visc_dissipation"
    rows = np.array([[float(v) for v in line.split(",")] for line in lines[1:]])
    assert rows.shape == (101, 6)
    assert np.array_equal(rows[:, 0], np.arange(3, 104))
    assert np.allclose(rows[:, 1], (3 + np.arange(101)) * dt, rtol=0, atol=1e-15)
    assert np.array_equal(rows[:, 2], ke) and np.array_equal(rows[:, 3], ens)
    assert np.max(np.abs(rows[1:-1, 4] - 0.0625 * np.exp(-0.5 * t[1:-1]))) < 1e-5
    assert np.allclose(rows[:, 5], 2.0 * ens / Re, rtol=1e-15)
    one = tmp_path / "one.csv"
    ex.write_series_csv(str(one), ke[:1], ens[:1], dt, Re)
    assert one.read_text().splitlines()[1].split(",")[4] == ""

"""GPU scalar advection-diffusion (osb_scalar_rk3) against the oracle and the
paper's verification results: the Section 3.1 wave (eighth order, Courant
0.2, error O(1e-10) at t = 1) and the Section 3.2 manufactured solution
(steady error slopes equal to the scheme order, 2..12).  FP64, held to the
1e-12 bar against the oracle."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import oracle as orc
from tests.test_scalar_oracle import MMS, _wave_case, mms_discrete_steady, mms_source

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01277_gb300 import build
    build.build()
    from paper_1609_01277_gb300 import osb
    osb.load()
    return osb, torch


def _gpu_run(env, phi0, order, adv, k, dt, nsteps, S=None, chunks=None):
    osb, torch = env
    phi = torch.from_numpy(np.ascontiguousarray(phi0, dtype=np.float64)).cuda()
    work = torch.empty(2 * phi.numel(), dtype=torch.float64, device="cuda")
    src = None if S is None else torch.from_numpy(np.ascontiguousarray(S, dtype=np.float64)).cuda()
    for n in (chunks or [nsteps]):
        osb.scalar_rk3(phi, work, order, adv, k, dt, n, src)
    torch.cuda.synchronize()
    return phi.cpu().numpy()


def test_wave_matches_oracle_and_paper_error(env):
    w, n, steps, a = _wave_case()
    x = np.arange(n) * 2 * math.pi / n
    phi0 = np.sin(x).reshape(1, 1, n)
    g = _gpu_run(env, phi0, w["order"], (a, 0, 0), 0.0, w["dt"], steps).ravel()
    o = orc.scalar_rk3(orc.Case(n, 1, 1, order=w["order"], dt=w["dt"]), phi0, adv=(a, 0, 0), nsteps=steps).ravel()
    assert np.max(np.abs(g - o)) < 1e-12
    err = np.max(np.abs(g - np.sin(x - a * w["t_end"])))
    mag = w["error_order_of_magnitude"]
    assert mag / 10 <= err <= mag * 10, err


def _mms_gpu(env, order, n, t_end=25.0, cfl=0.025):
    h = 2 * math.pi / n
    dt = cfl * h / max(abs(v) for v in MMS["u"])
    steps = int(math.ceil(t_end / dt))
    return _gpu_run(env, np.zeros((1, n, n)), order, (MMS["u"][0], MMS["u"][1], 0.0), MMS["k"], dt, steps,
                    S=mms_source(n)), dt, steps


@pytest.mark.parametrize("order,n", [(2, 16), (4, 16), (8, 32), (12, 32)])
def test_mms_matches_oracle_and_discrete_steady_state(env, order, n):
    g, dt, steps = _mms_gpu(env, order, n)
    o = orc.scalar_rk3(orc.Case(n, n, 1, order=order, dt=dt), np.zeros((1, n, n)),
                       adv=(MMS["u"][0], MMS["u"][1], 0.0), k=MMS["k"], S=mms_source(n), nsteps=steps)
    assert np.max(np.abs(g - o)) < 1e-12
    assert np.max(np.abs(g - mms_discrete_steady(order, n))) < 1e-11


def test_mms_convergence_slopes_on_gpu(env):
    """The paper's Figure of steady errors: slope = order for orders 2..12."""
    for order in (2, 4, 6, 8, 10, 12):
        errs = []
        for n in (8, 16, 32, 64):
            g, _, _ = _mms_gpu(env, order, n)
            x = np.arange(n) * 2 * math.pi / n
            X0, X1 = np.meshgrid(x, x, indexing="xy")
            errs.append(float(np.sqrt(np.mean((g[0] - np.sin(X0) * np.cos(X1)) ** 2))))
        pts = [(n, e) for n, e in zip((8, 16, 32, 64), errs) if e > 1e-12]
        slope = math.log(pts[-2][1] / pts[-1][1], 2)
        assert abs(slope - order) < 0.35, (order, errs)


def test_3d_ragged_anisotropic_matches_oracle(env):
    nx, ny, nz = 20, 12, 9
    rng = np.random.default_rng(7)
    x = [np.arange(m) * 2 * math.pi / m for m in (nx, ny, nz)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    phi0 = np.sin(X + 0.3) * np.cos(2 * Y) + 0.5 * np.cos(Z - X) + 0.1 * rng.standard_normal((nz, ny, nx))
    S = 0.2 * np.cos(X) * np.sin(Y + Z)
    adv, k, dt, steps = (0.3, -0.7, 1.1), 0.05, 2e-3, 7
    g = _gpu_run(env, phi0, 6, adv, k, dt, steps, S=S)
    o = orc.scalar_rk3(orc.Case(nx, ny, nz, order=6, dt=dt), phi0, adv=adv, k=k, S=S, nsteps=steps)
    assert np.linalg.norm(g - o) / np.linalg.norm(o) < 1e-12


def test_step_splitting_is_bitwise(env):
    """Odd and even step counts leave the result in the caller's array; 3 + 2
    steps give the bits of 5 (the register roles alternate per step)."""
    n = 24
    rng = np.random.default_rng(3)
    phi0 = rng.standard_normal((n, n, n))
    a = _gpu_run(env, phi0, 4, (0.5, 0.25, -1.0), 0.01, 1e-3, 5)
    b = _gpu_run(env, phi0, 4, (0.5, 0.25, -1.0), 0.01, 1e-3, 5, chunks=[3, 2])
    c = _gpu_run(env, phi0, 4, (0.5, 0.25, -1.0), 0.01, 1e-3, 5, chunks=[1, 1, 1, 1, 1])
    assert np.array_equal(a, b) and np.array_equal(a, c)

"""Forward Euler (osb_euler_step, Section 2.4) on the GPU against the oracle:
FP64 to the 1e-12 bar, FP32 to the FP32 bound; mixed with RK3 steps."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs
from tests.helpers import conserved

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
    return m


def _errs(Q, ref):
    mnorm = np.linalg.norm(ref[1:4].ravel())
    return [float(np.linalg.norm((Q[m] - ref[m]).ravel()) /
                  (mnorm if 1 <= m <= 3 else np.linalg.norm(ref[m].ravel()))) for m in range(5)]


@pytest.mark.parametrize("shape,order", [((16, 16, 16), 4), ((12, 10, 14), 8)])
def test_euler_fp64_matches_oracle(osb, shape, order):
    nx, ny, nz = shape
    case = orc.Case(nx, ny, nz, order=order, dt=1e-3)
    Q0 = conserved(*inputs.smooth_primitive_state(nx, ny, nz, seed=17), gamma=case.gamma)
    g = osb.Grid(osb.Config(nx, ny, nz, order=order, dt=1e-3))
    g.set_state(Q0)
    g.euler_step(5)
    assert max(_errs(g.get_state(), orc.euler_step(case, Q0, 5))) < 1e-12
    assert g.diagnostics()["step"] == 5


def test_euler_and_rk3_mix(osb):
    n = 16
    case = orc.Case(n, n, n, order=4, dt=1e-3)
    Q0 = orc.tgv_init(case, inputs.gaussian_noise(n, n, n, 9), 1e-3)
    ref = orc.rk3_step(case, orc.euler_step(case, Q0, 2), 3)
    ref = orc.euler_step(case, ref, 1)
    for prec, tol in ((osb.OSB_FP64, 1e-12), (osb.OSB_FP32, 1e-5)):
        g = osb.Grid(osb.Config(n, n, n, order=4, precision=prec, dt=1e-3))
        g.set_state(Q0)
        g.euler_step(2)
        g.step(3)
        g.euler_step(1)
        assert max(_errs(g.get_state(), ref)) < tol, prec

"""The FP32 path's error per conserved field after a longer run, on the order-8
Taylor-Green case at 64^3 (the CPU-sized companion of the 512^3 order-8 FP32
run): 200 steps of the FP64 and FP32 GPU paths against the oracle.

FP64 is held to the 1e-12 bar.  FP32 keeps FP64 only in the RK accumulator
and the reductions.  The largest FP32 term is the pressure gradient at low
Mach number: p ~ 1/(gamma M^2) = 71 and rho E ~ 179, so FP32 rounding (6e-8)
leaves ~1e-5 absolute in p, and the first-derivative stencil (weights summing
in magnitude to ~1.4/h, h = 2 pi/64) makes that ~1e-4 in the momentum
residual.  The accumulator adds beta_k dt of it per stage; with rounding
errors uncorrelated between stages the momentum error after n steps is about
dt * 1e-4 * sqrt(n * sum_k beta_k^2) = 3.4e-3 * 1e-4 * 9.4 = 3.2e-6, i.e.
~6e-6 relative to |rho u| ~ 0.5.  Density and energy see only the smaller
convective terms.  The test allows 1e-5 and prints the measured values."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs

pytestmark = pytest.mark.gpu

N, ORDER, STEPS, DT = 64, 8, 200, 3.385e-3
FIELDS = ("rho", "rho_u", "rho_v", "rho_w", "rho_E")


@pytest.fixture(scope="module")
def runs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01277_gb300 import build
    build.build()
    from paper_1609_01277_gb300 import osb
    osb.load()
    noise = inputs.gaussian_noise(N, N, N, 1234)
    case = orc.Case(N, N, N, order=ORDER, dt=DT)
    Qo = orc.rk3_step(case, orc.tgv_init(case, noise, 1e-4), STEPS)
    out = {"oracle": Qo}
    for name, prec in (("fp64", osb.OSB_FP64), ("fp32", osb.OSB_FP32)):
        g = osb.Grid(osb.Config(N, N, N, order=ORDER, precision=prec, dt=DT))
        g.init_taylor_green(noise, 1e-4)
        g.step(STEPS)
        out[name] = g.get_state()
    return out


def _errors(Q, ref):
    mnorm = np.linalg.norm(ref[1:4].ravel())
    errs = {}
    for m, f in enumerate(FIELDS):
        scale = mnorm if 1 <= m <= 3 else np.linalg.norm(ref[m].ravel())
        errs[f] = float(np.linalg.norm((Q[m] - ref[m]).ravel()) / scale)
    return errs


def test_fp64_matches_oracle_after_200_steps(runs):
    e = _errors(runs["fp64"], runs["oracle"])
    print("FP64 vs oracle, 64^3 order 8, 200 steps:", e)
    assert max(e.values()) < 1e-12


def test_fp32_error_per_field_after_200_steps(runs):
    e_or = _errors(runs["fp32"], runs["oracle"])
    e_64 = _errors(runs["fp32"], runs["fp64"])
    print("FP32 vs oracle, 64^3 order 8, 200 steps:", e_or)
    print("FP32 vs FP64 GPU, 64^3 order 8, 200 steps:", e_64)
    assert max(e_or.values()) < 1e-5
    assert max(e_64.values()) < 1e-5

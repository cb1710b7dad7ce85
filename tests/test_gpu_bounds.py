"""The bounds-check build (-DOSB_BOUNDS_CHECK; compute-sanitizer is closed on
this pool): every index a stage kernel forms is tested against its buffer and
a failure is recorded in the grid's device error word, which osb_diagnostics
reports as OSB_ERR_BOUNDS.  Every stage path -- FP64, double-float, FP32 fused,
two-kernel and three-kernel, TMA and cp.async loads, viscous form B, forward
Euler, symmetry planes, z slabs with halo exchange, ensembles -- runs on
small, ragged and degenerate grids without a single violation, and the check
build still computes the oracle's state."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_check_build_reports_no_violation_on_any_path():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-m", "tests.bounds_run"], cwd=ROOT, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    state = np.array(out.pop("_state"))
    bad = {k: v for k, v in out.items() if v != 0}
    assert not bad, bad
    assert len(out) == 62
    case = orc.Case(13, 11, 9, order=4, Re=300.0, dt=1e-3)
    Qo = orc.rk3_step(case, orc.tgv_init(case, inputs.gaussian_noise(13, 11, 9, seed=33), 1e-3), 3)
    for m in range(5):
        scale = np.linalg.norm(Qo[1:4].ravel()) if 1 <= m <= 3 else np.linalg.norm(Qo[m].ravel())
        assert np.linalg.norm((state[m] - Qo[m]).ravel()) / scale < 1e-12, m

"""The allocation-free diagnostics entry point, through the C ABI, against the
regular osb_diagnostics on the same states, two calls in a row.

Some callers cannot allocate device memory where they need diagnostics (for
example inside a global-mode stream capture, where cudaMalloc is an error);
osb_diagnostics_noalloc serves them from a fixed array inside the library.
This file is collected last on purpose, and must pass both on its own in a
fresh process (the first call on the device looks up the array's address)
and after every other test."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1609_01277_gb300 import inputs

pytestmark = pytest.mark.gpu

REL = 1e-13  # the tolerance the diagnostics parity tests use


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


def _compare(out, ref):
    vals = out.cpu().numpy()
    expect = [ref["ke"], ref["enstrophy"], *ref["total"]]
    for got, want in zip(vals[:7], expect):
        assert got == pytest.approx(want, rel=REL, abs=1e-15)
    assert vals[7] == ref["nonfinite"]
    assert vals[8] == pytest.approx(ref["max_cfl"], rel=REL)


def test_noalloc_diagnostics_match_regular_diagnostics_twice(osb):
    import torch
    nx, ny, nz = 40, 24, 18
    cfg = osb.Config(nx, ny, nz, order=8, dt=1e-3)
    g = osb.Grid(cfg)
    g.init_taylor_green(inputs.gaussian_noise(nx, ny, nz, seed=99), 1e-2)
    L = osb.load()
    params = cfg.params()
    outs = []
    for call in range(2):
        if call == 1:
            g.step(3)  # a different state for the second call
        ref = g.diagnostics()
        Q = g.get_state_device()
        out = torch.full((9,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.osb_diagnostics_noalloc(Q.data_ptr(), nx, ny, nz, cfg.order, ctypes.byref(params),
                                       out.data_ptr(), g.stream.cuda_stream)
        assert st == 0, L.osb_last_error()
        torch.cuda.synchronize()
        _compare(out, ref)
        outs.append(out.cpu().numpy())
    assert not np.array_equal(outs[0], outs[1])

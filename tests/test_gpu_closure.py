"""Learned closure on the GPU against the CPU network oracle, through the C
ABI: forward, loss and parameter gradients, Adam, box filter, the correction
added to R, and what training gains over the solver without it.

Tolerances: the oracle rounds operands and activations to BF16 where the
kernels do, so what remains is FP32 accumulation on the GPU against float64
sums on the CPU, and the rare element whose pre-activation sits at a BF16
rounding boundary and rounds the other way.  Measured on 8 to 32 points per
axis: forward <= 6.5e-4, parameter gradients <= 3.8e-4, loss <= 2.7e-5
(relative L2); held to 3e-3, 3e-3 and 2e-4.  Grids whose y extent is a
multiple of 16 run the tcgen05 convolutions, the others the mma.sync tiles:
both are covered."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import closure_oracle as co
from oracle import oracle as orc
from paper_1609_01277_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01277_gb300 import build
    build.build()
    from paper_1609_01277_gb300 import closure, osb
    osb.load()
    return osb, closure, torch


def _setup(mods, n=(16, 8, 8), seed=0):
    osb, closure, torch = mods
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = (closure.init_params(seed) + rng.standard_normal(co.param_count()).astype(np.float32) * 0.02)
    theta = theta.astype(np.float32)
    Q = np.stack([1 + 0.2 * inputs.smooth_field(nx, ny, nz, seed + i) for i in range(5)])
    C = np.stack([inputs.smooth_field(nx, ny, nz, seed + 10 + i) for i in range(5)])
    mean, std, out = np.array([1.0, 0.9, 1.1, 1.0, 1.05]), np.array([0.2, 0.25, 0.2, 0.3, 0.2]), np.array(
        [0.5, 1.0, 2.0, 0.7, 1.5])
    c = closure.Closure(nx, ny, nz, params=theta)
    c.set_normalization(mean, std, out)
    return c, theta, Q, C, mean, std, out


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


FWD_TOL, GRAD_TOL, LOSS_TOL = 3e-3, 3e-3, 2e-4
SHAPES = [(16, 8, 8), (16, 16, 8), (24, 32, 8)]   # mma.sync tiles; tcgen05 (y multiple of 16)


@pytest.mark.parametrize("n", SHAPES)
def test_forward_matches_oracle(mods, n):
    osb, closure, torch = mods
    c, theta, Q, _, mean, std, out = _setup(mods, n=n)
    Cg = c.forward(torch.from_numpy(Q).cuda()).cpu().numpy()
    Co = co.correction(theta.astype(np.float64), Q, mean, std, out, mode="bf16")
    assert _rel(Cg, Co) < FWD_TOL


def test_dissipative_forward_matches_oracle(mods):
    osb, closure, torch = mods
    c, theta, Q, _, mean, std, out = _setup(mods)
    c.set_dissipative(True)
    try:
        Cg = c.forward(torch.from_numpy(Q).cuda()).cpu().numpy()
    finally:
        c.set_dissipative(False)
    Co = co.correction(theta.astype(np.float64), Q, mean, std, out, mode="bf16", dissipative=True)
    assert _rel(Cg, Co) < FWD_TOL
    u = Q[1:4] / Q[0]
    dg = np.sum(u * Cg[1:4].astype(np.float64), axis=0)
    assert np.all(dg <= 1e-5 * np.sum(np.abs(u * Cg[1:4]), axis=0) + 1e-30)


@pytest.mark.parametrize("n", [(16, 8, 12), (16, 16, 8), (32, 16, 12)])
def test_loss_and_gradients_match_oracle(mods, n):
    osb, closure, torch = mods
    c, theta, Q, C, mean, std, out = _setup(mods, n=n, seed=3)
    loss, grad = c.loss_grad(torch.from_numpy(Q).cuda(), torch.from_numpy(C).cuda())
    lo, go = co.loss_grad(theta.astype(np.float64), Q, C, mean, std, out, mode="bf16")
    assert float(loss.item()) == pytest.approx(lo, rel=LOSS_TOL)
    g = grad.cpu().numpy().astype(np.float64)
    P, Po = co.unpack(g), co.unpack(go)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert _rel(P[name], Po[name]) < GRAD_TOL, name


def test_loss_weight_scales_loss_and_gradient(mods):
    osb, closure, torch = mods
    c, theta, Q, C, *_ = _setup(mods, n=(16, 8, 12), seed=3)
    Qd, Cd = torch.from_numpy(Q).cuda(), torch.from_numpy(C).cuda()
    l1, g1 = c.loss_grad(Qd, Cd)       # the closure's own output buffers: copy before the next call
    l1 = float(l1.item())
    g1 = g1.cpu().numpy().astype(np.float64)
    c.set_loss_weight(4.0)   # a power of two: the BF16 output gradient scales exactly
    try:
        l4, g4 = c.loss_grad(Qd, Cd)
    finally:
        c.set_loss_weight(1.0)
    assert float(l4.item()) == pytest.approx(4.0 * l1, rel=1e-6)
    assert _rel(g4.cpu().numpy().astype(np.float64), 4.0 * g1) < 1e-5


def test_adam_step_matches_formula(mods):
    osb, closure, torch = mods
    c, theta, Q, C, *_ = _setup(mods, seed=5)
    Qd, Cd = torch.from_numpy(Q).cuda(), torch.from_numpy(C).cuda()
    _, grad = c.loss_grad(Qd, Cd)
    g = grad.cpu().numpy().astype(np.float64)
    c.train_step(Qd, Cd, 1e-3)
    th, _, _ = co.adam(theta.astype(np.float64), np.zeros_like(g), np.zeros_like(g), g, 1e-3, 1)
    assert np.allclose(c.get_params(), th, rtol=1e-5, atol=1e-7)


def test_box_filter_matches_oracle(mods):
    osb, closure, torch = mods
    rng = np.random.Generator(np.random.PCG64(4))
    Q = rng.standard_normal((5, 16, 8, 24))
    F = closure.box_filter(torch.from_numpy(Q).cuda(), (24, 8, 16), 4).cpu().numpy()
    assert np.allclose(F, co.box_filter(Q, 4), rtol=1e-14, atol=1e-15)


def test_attached_closure_adds_correction_to_residual(mods):
    osb, closure, torch = mods
    n = 16
    c, *_ = _setup(mods, n=(n, n, n), seed=7)
    g = osb.Grid(osb.Config(n, n, n, order=4, dt=1e-3))
    g.init_taylor_green(inputs.gaussian_noise(n, n, n, 1), 1e-2)
    R0 = g.residual().cpu().numpy()
    Cg = c.forward(g.get_state_device()).cpu().numpy().astype(np.float64)
    c.attach(g)
    R1 = g.residual().cpu().numpy()
    assert np.allclose(R1 - R0, Cg, rtol=1e-6, atol=1e-12 * np.abs(R0).max())
    # stepping with the closure differs; detaching restores the plain solver bitwise
    g.step(2)
    closure.Closure.detach(g)
    p = osb.Grid(osb.Config(n, n, n, order=4, dt=1e-3))
    p.set_state(g.get_state())
    q = osb.Grid(osb.Config(n, n, n, order=4, dt=1e-3))
    q.set_state(g.get_state())
    p.step(3)
    q.step(3)
    assert np.array_equal(p.get_state(), q.get_state())


def test_closure_in_fp32_order8_steps_narrow_and_wide_residual_kernels(mods, monkeypatch):
    """FP32 order-8 steps add the closure inside the z-march residual kernels
    (narrow by default, the 32x8 one with OSB_FP32_ZRHS=wide): the two agree
    to FP32 rounding, and both differ from the plain step by far more."""
    osb, closure, torch = mods
    n = 32
    c, *_ = _setup(mods, n=(n, n, n), seed=29)
    noise = inputs.gaussian_noise(n, n, n, 3)
    out = {}
    for mode, attach in (("narrow", True), ("wide", True), ("narrow", False)):
        monkeypatch.setenv("OSB_FP32_ZRHS", mode)
        g = osb.Grid(osb.Config(n, n, n, order=8, precision=osb.OSB_FP32, dt=1e-3))
        g.init_taylor_green(noise, 1e-2)
        if attach:
            c.attach(g)
        g.step(2)
        out[(mode, attach)] = g.get_state()
    a, b, plain = out[("narrow", True)], out[("wide", True)], out[("narrow", False)]
    scale = np.linalg.norm((a - plain).ravel())
    assert scale > 1e-8 * np.linalg.norm(plain.ravel())
    assert np.linalg.norm((a - b).ravel()) < 1e-3 * scale
    c.status()


def test_training_reduces_a_priori_error(mods):
    """Closure data from the solver (fine 64^3 -> coarse 16^3, factor 4): after
    training, the closure explains part of the commutation residual on held-out
    snapshots, which the plain coarse solver misses entirely (error 1)."""
    osb, closure, torch = mods
    data = closure.make_training_data(64, 4, snapshots=12, every=25, Re=400.0)
    c = closure.Closure(16, 16, 16, seed=0)
    c.set_normalization(*closure.normalisation(data))
    train_idx, test_idx = list(range(0, 12, 3)) + list(range(1, 12, 3)), list(range(2, 12, 3))
    base = closure.a_priori_error(None, data, test_idx)
    hist = closure.train(c, data, epochs=25, lr=2e-3, train_idx=train_idx)
    after = closure.a_priori_error(c, data, test_idx)
    assert base == pytest.approx(1.0)
    assert hist[-1] < 0.5 * hist[0]
    assert after < 0.8, (after, hist[:3], hist[-3:])


def test_tensor_core_convolutions_match_oracle(mods):
    """Grids with ny a multiple of 16 take the tcgen05 path (TMEM accumulator)
    for the 32-channel convolutions: forward and every gradient block vs the
    CPU oracle, and no accumulator wait ran out."""
    osb, closure, torch = mods
    c, theta, Q, C, mean, std, out = _setup(mods, n=(16, 16, 8), seed=11)
    Qd, Cd = torch.from_numpy(Q).cuda(), torch.from_numpy(C).cuda()
    Cg = c.forward(Qd).cpu().numpy()
    assert _rel(Cg, co.correction(theta.astype(np.float64), Q, mean, std, out, mode="bf16")) < FWD_TOL
    loss, grad = c.loss_grad(Qd, Cd)
    lo, go = co.loss_grad(theta.astype(np.float64), Q, C, mean, std, out, mode="bf16")
    assert float(loss.item()) == pytest.approx(lo, rel=LOSS_TOL)
    P, Po = co.unpack(grad.cpu().numpy().astype(np.float64)), co.unpack(go)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert _rel(P[name], Po[name]) < GRAD_TOL, name
    c.status()


def test_tensor_core_and_mma_sync_paths_agree(mods, monkeypatch):
    osb, closure, torch = mods
    c, theta, Q, C, *_ = _setup(mods, n=(32, 16, 4), seed=13)
    Qd = torch.from_numpy(Q).cuda()
    monkeypatch.setenv("OSB_CLOSURE_MMA", "sync")
    ref = c.forward(Qd).cpu().numpy()
    monkeypatch.setenv("OSB_CLOSURE_MMA", "tc")
    tc = c.forward(Qd).cpu().numpy()
    c.status()
    assert _rel(tc, ref) < 5e-3


@pytest.mark.parametrize("zchunk", ["1", "3", "5"])
def test_z_marching_tensor_core_chunks(mods, monkeypatch, zchunk):
    """The z-marching tcgen05 convolutions over z chunks of 1, 3 (ragged last
    chunk of 2) and 5 (3) planes agree bit for bit with one chunk of all 8
    planes (the same MMAs per accumulator), and with the CPU oracle."""
    osb, closure, torch = mods
    c, theta, Q, C, mean, std, out = _setup(mods, n=(16, 32, 8), seed=17)
    Qd, Cd = torch.from_numpy(Q).cuda(), torch.from_numpy(C).cuda()
    monkeypatch.setenv("OSB_CLOSURE_MMA", "tc")
    monkeypatch.setenv("OSB_TC_ZCHUNK", "8")
    ref = c.forward(Qd).cpu().numpy()
    lr, gr = c.loss_grad(Qd, Cd)
    lr, gr = float(lr.item()), gr.cpu().numpy()
    monkeypatch.setenv("OSB_TC_ZCHUNK", zchunk)
    got = c.forward(Qd).cpu().numpy()
    lt, gt = c.loss_grad(Qd, Cd)
    c.status()
    assert np.array_equal(got, ref)
    assert float(lt.item()) == pytest.approx(lr, rel=1e-6)
    assert _rel(gt.cpu().numpy(), gr) < 1e-6
    assert _rel(got, co.correction(theta.astype(np.float64), Q, mean, std, out, mode="bf16")) < FWD_TOL


def test_brick_and_z_marching_tensor_core_kernels_agree(mods, monkeypatch):
    """One brick per CTA (hidden layers on tcgen05, output layer on mma.sync)
    against the z-marching kernels (all three layers on tcgen05)."""
    osb, closure, torch = mods
    c, theta, Q, C, *_ = _setup(mods, n=(16, 32, 8), seed=19)
    Qd = torch.from_numpy(Q).cuda()
    monkeypatch.setenv("OSB_CLOSURE_MMA", "brick")
    ref = c.forward(Qd).cpu().numpy()
    monkeypatch.setenv("OSB_CLOSURE_MMA", "tc")
    got = c.forward(Qd).cpu().numpy()
    c.status()
    assert _rel(got, ref) < 1e-5


@pytest.mark.parametrize("zchunk", ["1", "4"])
@pytest.mark.parametrize("n", [(8, 16, 4), (24, 16, 4)])
def test_z_marching_convolutions_on_the_shallowest_grids(mods, monkeypatch, n, zchunk):
    """Four planes, the fewest a closure grid takes (its bricks are 4 deep):
    every window wraps in z, and a one-plane chunk loads the same planes into
    several ring slots.  Forward and gradients against the CPU oracle, and no
    accumulator wait ran out."""
    osb, closure, torch = mods
    c, theta, Q, C, mean, std, out = _setup(mods, n=n, seed=23)
    Qd, Cd = torch.from_numpy(Q).cuda(), torch.from_numpy(C).cuda()
    monkeypatch.setenv("OSB_CLOSURE_MMA", "tc")
    monkeypatch.setenv("OSB_TC_ZCHUNK", zchunk)
    Cg = c.forward(Qd).cpu().numpy()
    assert _rel(Cg, co.correction(theta.astype(np.float64), Q, mean, std, out, mode="bf16")) < FWD_TOL
    loss, grad = c.loss_grad(Qd, Cd)
    lo, go = co.loss_grad(theta.astype(np.float64), Q, C, mean, std, out, mode="bf16")
    assert float(loss.item()) == pytest.approx(lo, rel=LOSS_TOL)
    P, Po = co.unpack(grad.cpu().numpy().astype(np.float64)), co.unpack(go)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert _rel(P[name], Po[name]) < GRAD_TOL, name
    c.status()

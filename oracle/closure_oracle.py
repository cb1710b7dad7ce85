"""CPU oracle of the learned-closure network and of the box filter.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only the tests import this module.  It
shares nothing with the CUDA library.

Network (a learned closure; not in the paper): three 3x3x3 periodic
cross-correlations 5 -> 32 -> 32 -> 5 with ReLU after the first two,
    z(p) = b + sum_k W[:, :, k] x(p + off_k),  off_k = (dx, dy, dz),
    k = (dz+1)*9 + (dy+1)*3 + (dx+1),
on normalised inputs x_c = (Q_c - mean_c)/std_c; loss = mean((y - t)^2) over
5 channels and all points, t = C*/out_std.

mode="bf16": operands rounded to bfloat16 where the tensor-core path rounds
them (inputs, weights, hidden activations, the output gradient and the
hidden-layer gradients), sums in float64.  mode="exact": float64 throughout,
for finite-difference checks of the backward pass.
"""
from __future__ import annotations

import numpy as np

H = 32
SHAPES = [("W1", (H, 5, 27)), ("b1", (H,)), ("W2", (H, H, 27)), ("b2", (H,)), ("W3", (5, H, 27)), ("b3", (5,))]


def param_count() -> int:
    return sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, s in SHAPES:
        n = int(np.prod(s))
        out[name] = theta[o:o + n].reshape(s)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even); returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    r = ((a >> 16) & 1) + 0x7FFF
    b = ((a + r) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def _offset(k):
    return k % 3 - 1, (k // 3) % 3 - 1, k // 9 - 1  # dx, dy, dz


def _shift(x, dx, dy, dz):
    """out[..., z, y, x] = x[..., z+dz, y+dy, x+dx] (periodic)."""
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


def conv(x, W, b=None):
    """x: (Cin, nz, ny, nx), W: (Cout, Cin, 27) -> (Cout, nz, ny, nx)."""
    out = np.zeros((W.shape[0],) + x.shape[1:])
    for k in range(27):
        out += np.einsum("oc,czyx->ozyx", W[:, :, k], _shift(x, *_offset(k)))
    if b is not None:
        out += b[:, None, None, None]
    return out


def conv_t(d, W):
    """Adjoint of conv in x: (Cout, ...) -> (Cin, ...)."""
    out = np.zeros((W.shape[1],) + d.shape[1:])
    for k in range(27):
        dx, dy, dz = _offset(k)
        out += np.einsum("oc,ozyx->czyx", W[:, :, k], _shift(d, -dx, -dy, -dz))
    return out


def wgrad(d, x):
    """dW[co, ci, k] = sum_p d[co](p) x[ci](p + off_k)."""
    out = np.zeros((d.shape[0], x.shape[0], 27))
    for k in range(27):
        out[:, :, k] = np.einsum("ozyx,czyx->oc", d, _shift(x, *_offset(k)))
    return out


def normalise(Q, mean, std):
    return (np.asarray(Q, np.float64) - np.asarray(mean)[:, None, None, None]) / np.asarray(std)[:, None, None, None]


def forward(theta, Q, mean, std, mode="bf16"):
    """Returns y (5, nz, ny, nx) and the activations needed by backward."""
    P = unpack(np.asarray(theta, np.float64))
    r = bf16 if mode == "bf16" else (lambda v: np.asarray(v, np.float64))
    f32 = (lambda v: np.asarray(v, np.float32).astype(np.float64)) if mode == "bf16" else r
    x0 = r(normalise(Q, mean, std))
    W1, W2, W3 = r(P["W1"]), r(P["W2"]), r(P["W3"])
    h1 = r(np.maximum(f32(conv(x0, W1, P["b1"])), 0.0))
    h2 = r(np.maximum(f32(conv(h1, W2, P["b2"])), 0.0))
    y = f32(conv(h2, W3, P["b3"]))
    return y, dict(x0=x0, h1=h1, h2=h2, W1=W1, W2=W2, W3=W3)


def loss_grad(theta, Q, Cstar, mean, std, out_std, mode="bf16"):
    """MSE loss on the normalised output and its gradient (flat, param layout)."""
    y, A = forward(theta, Q, mean, std, mode)
    t = np.asarray(Cstar, np.float64) / np.asarray(out_std)[:, None, None, None]
    if mode == "bf16":
        t = np.asarray(t, np.float32).astype(np.float64)
    n = y[0].size
    diff = y - t
    loss = float(np.mean(diff ** 2))
    r = bf16 if mode == "bf16" else (lambda v: np.asarray(v, np.float64))
    f32 = (lambda v: np.asarray(v, np.float32).astype(np.float64)) if mode == "bf16" else r
    dy = r(2.0 * f32(diff) / (5 * n))
    g = {"W3": wgrad(dy, A["h2"]), "b3": dy.sum(axis=(1, 2, 3))}
    dz2 = r(conv_t(dy, A["W3"]) * (A["h2"] > 0))
    g["W2"] = wgrad(dz2, A["h1"])
    g["b2"] = dz2.sum(axis=(1, 2, 3))
    dz1 = r(conv_t(dz2, A["W2"]) * (A["h1"] > 0))
    g["W1"] = wgrad(dz1, A["x0"])
    g["b1"] = dz1.sum(axis=(1, 2, 3))
    return loss, pack(g)


def correction(theta, Q, mean, std, out_std, mode="bf16", dissipative=False):
    """C = out_std * y.  dissipative: where the momentum part feeds kinetic
    energy (u . C_m > 0, u = m / rho) its component along u is removed."""
    y, _ = forward(theta, Q, mean, std, mode)
    C = y * np.asarray(out_std)[:, None, None, None]
    if dissipative:
        Q = np.asarray(Q, np.float64)
        u = Q[1:4] / Q[0]
        d = np.sum(u * C[1:4], axis=0)
        uu = np.sum(u * u, axis=0)
        s = np.where((d > 0) & (uu > 0), d / np.where(uu > 0, uu, 1.0), 0.0)
        C = C.copy()
        C[1:4] -= s * u
    return C


def adam(theta, m, v, g, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    c1, c2 = 1.0 / (1 - b1 ** step), 1.0 / (1 - b2 ** step)
    return theta - lr * (m * c1) / (np.sqrt(v * c2) + eps), m, v


def box_filter(Q, f):
    """Mean over f^3 blocks of each field: (5, nz, ny, nx) -> (5, nz/f, ny/f, nx/f)."""
    c, nz, ny, nx = Q.shape
    return Q.reshape(c, nz // f, f, ny // f, f, nx // f, f).mean(axis=(2, 4, 6))

"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the method (no stencil, residual, RK or
initial-condition formula).  It only draws random numbers and random smooth
fields from fixed seeds, so that both sides of a parity test start from the
same bytes:

* ``gaussian_noise`` -- the N(0,1) draws that perturb the Taylor-Green
  velocity components (three fields, ``[3][z][y][x]``);
* ``smooth_field`` -- a random periodic trigonometric polynomial, used to
  build arbitrary smooth states for parity and conservation tests;
* ``ensemble`` -- the uneven instance list of the batched ensemble workload.
"""
from __future__ import annotations

import numpy as np


def gaussian_noise(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """Three independent N(0,1) fields, float64, shape (3, nz, ny, nx)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((3, nz, ny, nx))


def smooth_field(nx: int, ny: int, nz: int, seed: int, modes: int = 3,
                 amp: float = 1.0) -> np.ndarray:
    """Random periodic field sum_k a_k cos(k.x + phi_k) on [0, 2pi)^3 with
    integer wavenumbers |k_i| <= modes; float64, shape (nz, ny, nx)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = 2.0 * np.pi * np.arange(nx) / nx
    y = 2.0 * np.pi * np.arange(ny) / ny
    z = 2.0 * np.pi * np.arange(nz) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = np.zeros((nz, ny, nx))
    nterms = 6
    for _ in range(nterms):
        k = rng.integers(-modes, modes + 1, size=3)
        a = rng.uniform(-1.0, 1.0) * amp / nterms
        phi = rng.uniform(0.0, 2.0 * np.pi)
        f += a * np.cos(k[0] * X + k[1] * Y + k[2] * Z + phi)
    return f


def smooth_primitive_state(nx: int, ny: int, nz: int, seed: int):
    """Random smooth primitive fields (rho, u0, u1, u2, p) of a subsonic
    compressible flow: rho, p positive, |u| of order one."""
    rho = 1.0 + 0.3 * smooth_field(nx, ny, nz, seed + 1)
    u = [smooth_field(nx, ny, nz, seed + 2 + i) for i in range(3)]
    p = 71.43 + 5.0 * smooth_field(nx, ny, nz, seed + 5)
    return rho, u[0], u[1], u[2], p


def ensemble(count: int, seed: int, sizes=(32, 48, 64, 96, 128),
             re_range=(100.0, 3200.0), mach_range=(0.05, 0.3)):
    """Uneven Taylor-Green ensemble: per instance a cubic grid size drawn
    uniformly from ``sizes``, Re and Mach uniform in their ranges."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.choice(np.asarray(sizes), size=count)
    re = rng.uniform(*re_range, size=count)
    mach = rng.uniform(*mach_range, size=count)
    return [dict(n=int(n[i]), Re=float(re[i]), Mach=float(mach[i])) for i in range(count)]


def ensemble_with_dt(count: int = 64, seed: int = 7, base_dt_64: float = 3.385e-3):
    """The uneven ensemble with a time step per instance: the 64^3, M = 0.1
    step scaled by 64/N and by 11/(1 + 1/M), which keeps the acoustic Courant
    number of that case (sound speed ~ 1/M, flow speed ~ 1)."""
    out = []
    for e in ensemble(count, seed):
        e["dt"] = base_dt_64 * (64.0 / e["n"]) * 11.0 / (1.0 + 1.0 / e["Mach"])
        out.append(e)
    return out

"""ctypes wrapper around the CPU oracle (``osb_oracle.c``).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark import this module.  It shares nothing with
the CUDA library and never calls it.

Every array is a C-contiguous float64 numpy array in the layout
``[field][z][y][x]`` (x fastest), fields ``(rho, rho*u0, rho*u1, rho*u2, rho*E)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "osb_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP over z)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("order", ctypes.c_int), ("visc_form", ctypes.c_int),
                ("Re", ctypes.c_double), ("Mach", ctypes.c_double), ("gamma", ctypes.c_double),
                ("Pr", ctypes.c_double), ("dt", ctypes.c_double), ("nz_domain", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = P(ctypes.c_double)
        g = P(_Grid)
        _lib.orc_fd_coeffs.argtypes = [ctypes.c_int, d, d]
        _lib.orc_d1.argtypes = [g, ctypes.c_int, d, d]
        _lib.orc_d2.argtypes = [g, ctypes.c_int, d, d]
        _lib.orc_primitives.argtypes = [g, d, d, d, d]
        _lib.orc_residual.argtypes = [g, d, d]
        _lib.orc_rk3_step.argtypes = [g, d, ctypes.c_int]
        _lib.orc_rk3_coeffs.argtypes = [d, d]
        _lib.orc_rk3_linear.argtypes = [ctypes.c_size_t, d, d, ctypes.c_int, ctypes.c_double]
        _lib.orc_scalar_rk3.argtypes = [g, d, ctypes.c_double, d, d, ctypes.c_int]
        _lib.orc_euler_step.argtypes = [g, d, ctypes.c_int]
        _lib.orc_euler_linear.argtypes = [ctypes.c_size_t, d, d, ctypes.c_int, ctypes.c_double]
        _lib.orc_tgv_init.argtypes = [g, d, ctypes.c_double, d]
        _lib.orc_diagnostics.argtypes = [g, d, d]
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib.orc_get_threads.restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Case:
    """Grid and physical parameters (Section 3.3 defaults: Re 1600, M 0.1,
    gamma 1.4, Pr 0.71, dt 3.385e-3)."""
    nx: int
    ny: int
    nz: int
    order: int = 4
    visc_form: int = 0
    Re: float = 1600.0
    Mach: float = 0.1
    gamma: float = 1.4
    Pr: float = 0.71
    dt: float = 3.385e-3
    nz_domain: int = 0  # z-slab of a periodic grid with this many planes (0: the array is the grid)

    def c(self) -> _Grid:
        return _Grid(self.nx, self.ny, self.nz, self.order, self.visc_form,
                     self.Re, self.Mach, self.gamma, self.Pr, self.dt, self.nz_domain)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nx * self.ny * self.nz


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def fd_coeffs(order: int):
    r = order // 2
    c = np.zeros(7)
    d = np.zeros(7)
    if lib().orc_fd_coeffs(order, _p(c), _p(d)) != 0:
        raise ValueError(f"invalid order {order}")
    return c[: r + 1].copy(), d[: r + 1].copy()


def d1(case: Case, axis: int, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(case.shape)
    out = np.empty_like(f)
    g = case.c()
    lib().orc_d1(ctypes.byref(g), axis, _p(f), _p(out))
    return out


def d2(case: Case, axis: int, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(case.shape)
    out = np.empty_like(f)
    g = case.c()
    lib().orc_d2(ctypes.byref(g), axis, _p(f), _p(out))
    return out


def primitives(case: Case, Q: np.ndarray):
    Q = np.ascontiguousarray(Q, dtype=np.float64).reshape((5,) + case.shape)
    u = np.empty((3,) + case.shape)
    p = np.empty(case.shape)
    T = np.empty(case.shape)
    g = case.c()
    lib().orc_primitives(ctypes.byref(g), _p(Q), _p(u), _p(p), _p(T))
    return u, p, T


def residual(case: Case, Q: np.ndarray) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64).reshape((5,) + case.shape)
    R = np.empty_like(Q)
    g = case.c()
    if lib().orc_residual(ctypes.byref(g), _p(Q), _p(R)) != 0:
        raise MemoryError("oracle residual: allocation failed")
    return R


def rk3_step(case: Case, Q: np.ndarray, nsteps: int = 1) -> np.ndarray:
    Q = np.array(Q, dtype=np.float64, order="C").reshape((5,) + case.shape)
    g = case.c()
    if lib().orc_rk3_step(ctypes.byref(g), _p(Q), int(nsteps)) != 0:
        raise MemoryError("oracle rk3: allocation failed")
    return Q


def euler_step(case: Case, Q: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """Forward Euler (Section 2.4): Q^{n+1} = Q^n + dt R(Q^n)."""
    y = np.ascontiguousarray(Q, dtype=np.float64).reshape((5,) + case.shape).copy()
    g = case.c()
    if lib().orc_euler_step(ctypes.byref(g), _p(y), int(nsteps)) != 0:
        raise MemoryError("orc_euler_step")
    return y


def euler_linear(lam: np.ndarray, y0: np.ndarray, nsteps: int, dt: float) -> np.ndarray:
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    y = np.ascontiguousarray(y0, dtype=np.float64).copy()
    lib().orc_euler_linear(lam.size, _p(lam), _p(y), int(nsteps), float(dt))
    return y


def rk3_coeffs():
    a = np.zeros(3)
    b = np.zeros(3)
    lib().orc_rk3_coeffs(_p(a), _p(b))
    return a, b


def rk3_linear(lam: np.ndarray, y0: np.ndarray, nsteps: int, dt: float) -> np.ndarray:
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    y = np.array(y0, dtype=np.float64, order="C")
    lib().orc_rk3_linear(lam.size, _p(lam), _p(y), int(nsteps), float(dt))
    return y


def scalar_rk3(case: Case, phi: np.ndarray, adv=(0.0, 0.0, 0.0), k: float = 0.0, S: np.ndarray | None = None,
               nsteps: int = 1) -> np.ndarray:
    """Scalar advection-diffusion d phi/dt = -a_j D_j phi + k L_j phi - S
    (Sections 3.1 and 3.2) advanced nsteps RK3 steps of case.dt; phi and S are
    (nz, ny, nx) float64 arrays."""
    y = np.ascontiguousarray(phi, dtype=np.float64).reshape(case.shape).copy()
    a = np.ascontiguousarray(adv, dtype=np.float64)
    Sp = None
    if S is not None:
        S = np.ascontiguousarray(S, dtype=np.float64).reshape(case.shape)
        Sp = _p(S)
    g = case.c()
    if lib().orc_scalar_rk3(ctypes.byref(g), _p(a), float(k), Sp, _p(y), int(nsteps)) != 0:
        raise MemoryError("orc_scalar_rk3")
    return y


def tgv_init(case: Case, noise: np.ndarray | None = None, amp: float = 0.0) -> np.ndarray:
    Q = np.empty((5,) + case.shape)
    g = case.c()
    if noise is not None:
        noise = np.ascontiguousarray(noise, dtype=np.float64).reshape((3,) + case.shape)
        lib().orc_tgv_init(ctypes.byref(g), _p(noise), float(amp), _p(Q))
    else:
        lib().orc_tgv_init(ctypes.byref(g), None, 0.0, _p(Q))
    return Q


DIAG_KEYS = ("ke", "enstrophy", "rho", "rhou0", "rhou1", "rhou2", "rhoE", "nonfinite", "max_cfl")


def diagnostics(case: Case, Q: np.ndarray) -> dict:
    Q = np.ascontiguousarray(Q, dtype=np.float64).reshape((5,) + case.shape)
    out = np.zeros(9)
    g = case.c()
    lib().orc_diagnostics(ctypes.byref(g), _p(Q), _p(out))
    return dict(zip(DIAG_KEYS, out.tolist()))

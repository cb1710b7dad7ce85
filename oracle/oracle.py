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


# ---------------------------------------------------------------------------
# Symmetry boundaries (Section 2.6, "Boundary conditions").
#
# On an axis with symmetry planes the halo beyond the plane after the last
# point holds the mirror image of the points before it: a scalar field keeps
# its value, phi(x_{N+k}) = phi(x_{N-1-k}), and the component of a vector
# field along that axis changes sign.  The same rule applies at the first
# point, phi(x_{-1-k}) = phi(x_k).  The paper states the rule for the
# prognostic fields; every other quantity of the scheme (velocities, pressure,
# fluxes, their derivatives) is evaluated from those halos.  Applying the rule
# to the conserved fields therefore turns an N-point axis into the 2N-point
# periodic axis of the mirror-extended field, and the scheme on the symmetric
# grid is the periodic scheme on the extended grid restricted to the first N
# points.  The oracle below is exactly that: extend, run the periodic oracle,
# restrict.
#
# Coordinates: a periodic axis is [0, 2 pi) with x_i = i h, h = 2 pi / N; a
# symmetric axis lies between planes at 0 and pi with x_i = (i + 1/2) h,
# h = pi / N, so its 2N-point extension is a periodic [0, 2 pi) axis with the
# same spacing.
# ---------------------------------------------------------------------------

# sign of each conserved field (rho, rho u0, rho u1, rho u2, rho E) under the
# mirror across a plane normal to axis 0 (x), 1 (y), 2 (z)
SYM_PARITY = np.array([[1, 1, 1], [-1, 1, 1], [1, -1, 1], [1, 1, -1], [1, 1, 1]], dtype=np.float64)


def sym_extend(Q: np.ndarray, sym) -> np.ndarray:
    """Mirror-extend a (5, nz, ny, nx) state along every axis a with sym[a]
    (Section 2.6): the appended half is the reversed field times the field's
    parity for that axis."""
    Q = np.asarray(Q, dtype=np.float64)
    for a in range(3):
        if not sym[a]:
            continue
        arr_axis = 3 - a  # array layout [field][z][y][x]
        mirrored = np.flip(Q, axis=arr_axis) * SYM_PARITY[:, a].reshape(5, 1, 1, 1)
        Q = np.concatenate([Q, mirrored], axis=arr_axis)
    return np.ascontiguousarray(Q)


def sym_restrict(Qe: np.ndarray, case: Case) -> np.ndarray:
    """The first nx, ny, nz points of an extended field."""
    return np.ascontiguousarray(Qe[..., : case.nz, : case.ny, : case.nx])


def sym_case(case: Case, sym) -> Case:
    """The periodic case of the extended grid (2N points on symmetric axes,
    same spacing)."""
    from dataclasses import replace
    return replace(case, nx=case.nx * (2 if sym[0] else 1), ny=case.ny * (2 if sym[1] else 1),
                   nz=case.nz * (2 if sym[2] else 1))


def sym_residual(case: Case, Q: np.ndarray, sym) -> np.ndarray:
    return sym_restrict(residual(sym_case(case, sym), sym_extend(Q, sym)), case)


def sym_rk3_step(case: Case, Q: np.ndarray, nsteps: int, sym) -> np.ndarray:
    return sym_restrict(rk3_step(sym_case(case, sym), sym_extend(Q, sym), nsteps), case)


def sym_euler_step(case: Case, Q: np.ndarray, nsteps: int, sym) -> np.ndarray:
    return sym_restrict(euler_step(sym_case(case, sym), sym_extend(Q, sym), nsteps), case)


def axis_coords(n: int, symmetric: bool) -> np.ndarray:
    """Point coordinates of one axis (see the block comment above)."""
    i = np.arange(n, dtype=np.float64)
    return (i + 0.5) * (np.pi / n) if symmetric else i * (2.0 * np.pi / n)


def tgv_state(case: Case, sym=(False, False, False), noise: np.ndarray | None = None, amp: float = 0.0) -> np.ndarray:
    """Taylor-Green initial state (Section 3.3) at the grid's points, on
    periodic or symmetric axes; noise as in tgv_init."""
    return tgv_at(case, axis_coords(case.nx, sym[0]), axis_coords(case.ny, sym[1]), axis_coords(case.nz, sym[2]),
                  noise, amp)


def tgv_at(case: Case, x: np.ndarray, y: np.ndarray, z: np.ndarray, noise: np.ndarray | None = None,
           amp: float = 0.0) -> np.ndarray:
    """Taylor-Green initial state (Section 3.3, T = 1 so rho = gamma M^2 p) on
    the tensor grid of the coordinate vectors x, y, z (lengths nx, ny, nz)."""
    X = np.asarray(x, dtype=np.float64).reshape(1, 1, -1)
    Y = np.asarray(y, dtype=np.float64).reshape(1, -1, 1)
    Z = np.asarray(z, dtype=np.float64).reshape(-1, 1, 1)
    gM2 = case.gamma * case.Mach ** 2
    shape = case.shape
    u0 = np.broadcast_to(np.sin(X) * np.cos(Y) * np.cos(Z), shape).copy()
    u1 = np.broadcast_to(-np.cos(X) * np.sin(Y) * np.cos(Z), shape).copy()
    u2 = np.zeros(shape)
    p = np.broadcast_to(1.0 / gM2 + (np.cos(2 * X) + np.cos(2 * Y)) * (2.0 + np.cos(2 * Z)) / 16.0, shape)
    rho = gM2 * p
    if noise is not None:
        nz_ = np.asarray(noise, dtype=np.float64).reshape((3,) + shape)
        u0 += amp * nz_[0]
        u1 += amp * nz_[1]
        u2 += amp * nz_[2]
    return np.stack([rho, rho * u0, rho * u1, rho * u2,
                     p / (case.gamma - 1.0) + 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2)])


def sym_diagnostics(case: Case, Q: np.ndarray, sym) -> dict:
    """Diagnostics of Section 3.3 on a grid with symmetry planes: grid means
    over this grid's points.  The enstrophy's first derivatives and the CFL
    number come from the extended periodic grid; the kinetic energy,
    enstrophy, CFL and non-finite count are even under every mirror, so their
    extended-grid means equal the means here; the totals are plain means of
    this grid's fields."""
    d = diagnostics(sym_case(case, sym), sym_extend(Q, sym))
    Q = np.asarray(Q, dtype=np.float64).reshape((5,) + case.shape)
    for m, k in enumerate(("rho", "rhou0", "rhou1", "rhou2", "rhoE")):
        d[k] = float(Q[m].mean())
    d["nonfinite"] = float(np.count_nonzero(~np.isfinite(Q).all(axis=0)))
    return d

"""Small shared helpers for the tests (input construction and error norms).

Nothing here computes a residual, a stencil or a time step: it only turns
primitive input fields into the conserved layout both sides consume and
measures differences.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("rho", "rhou0", "rhou1", "rhou2", "rhoE")


def conserved(rho, u0, u1, u2, p, gamma=1.4) -> np.ndarray:
    """Pack primitive input fields into the conserved SoA state [5][z][y][x]."""
    e = p / (gamma - 1.0) + 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2)
    return np.ascontiguousarray(np.stack([rho, rho * u0, rho * u1, rho * u2, e]))


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2 (||b|| replaced by 1 when b is identically 0)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b.ravel()))
    return float(np.linalg.norm((a - b).ravel())) / (nb if nb > 0 else 1.0)


def rel_l2_fields(a: np.ndarray, b: np.ndarray) -> dict:
    return {FIELDS[m]: rel_l2(a[m], b[m]) for m in range(5)}

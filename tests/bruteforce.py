"""50-digit brute-force evaluation of the semi-discrete Navier-Stokes residual
and of the low-storage RK3 step on tiny periodic grids (8^3 and the like).

An independent second statement of the discretisation of Section 3.3 of the
OpenSBLI paper, written differently from the oracle on purpose:

* stencil weights come from solving the Taylor moment conditions exactly in
  rationals (not from the closed form the oracle uses);
* derivatives are dense circulant matrices applied along grid lines;
* arithmetic is ``decimal`` at 50 significant digits;
* the viscous momentum term uses the simplified algebra
  (1/Re)[sum_j L_j u_i + (1/3)(L_i u_i + sum_{k!=i} D_i D_k u_k)], which equals
  the term-by-term expansion of d_j tau_ij because tensor-product stencils
  along different axes commute.

Only +, -, *, / act on the state, so the input (exact binary64 values) is
carried without transcendental functions.
"""
from __future__ import annotations

from decimal import Decimal, getcontext
from fractions import Fraction

getcontext().prec = 50


# --------------------------------------------------------------------------
# Stencil weights by exact Taylor matching
# --------------------------------------------------------------------------
def _solve(A, b):
    """Gaussian elimination over Fractions."""
    n = len(A)
    M = [list(map(Fraction, row)) + [Fraction(v)] for row, v in zip(A, b)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col] / M[col][col]
                M[r] = [a - f * c for a, c in zip(M[r], M[col])]
    return [M[i][n] / M[i][i] for i in range(n)]


def first_derivative_weights(r: int):
    """Antisymmetric weights w_k (k = 1..r) with sum_k w_k (k^p - (-k)^p) = p! delta_{p1}
    for odd p = 1, 3, ..., 2r-1: the unique order-2r central first derivative."""
    A = [[2 * Fraction(k) ** p for k in range(1, r + 1)] for p in range(1, 2 * r, 2)]
    b = [1] + [0] * (r - 1)
    return _solve(A, b)


def second_derivative_weights(r: int):
    """Symmetric weights (w_0; w_1..w_r) with w_0 [p==0] + sum_k w_k 2 k^p = p! delta_{p2}
    for even p = 0, 2, ..., 2r."""
    A = []
    b = []
    for p in range(0, 2 * r + 1, 2):
        row = [Fraction(1 if p == 0 else 0)] + [2 * Fraction(k) ** p for k in range(1, r + 1)]
        A.append(row)
        b.append(2 if p == 2 else 0)
    w = _solve(A, b)
    return w[0], w[1:]


def pi_decimal() -> Decimal:
    """pi by Machin's formula, 16 atan(1/5) - 4 atan(1/239), at the context precision."""
    getcontext().prec += 5

    def atan_inv(x: int) -> Decimal:
        x = Decimal(x)
        x2 = x * x
        term = 1 / x
        s = term
        k = 1
        while True:
            term = -term / x2
            t = term / (2 * k + 1)
            if t == 0 or abs(t) < Decimal(10) ** (-(getcontext().prec + 2)):
                break
            s += t
            k += 1
        return s

    pi = 16 * atan_inv(5) - 4 * atan_inv(239)
    getcontext().prec -= 5
    return +pi


# --------------------------------------------------------------------------
# Dense circulant operators on a periodic box
# --------------------------------------------------------------------------
class Box:
    def __init__(self, nx, ny, nz, order):
        self.n = (nx, ny, nz)
        self.r = order // 2
        pi = pi_decimal()
        c = first_derivative_weights(self.r)
        d0, d = second_derivative_weights(self.r)
        self.D1 = []
        self.D2 = []
        for n in self.n:
            h = 2 * pi / n
            m1 = [[Decimal(0)] * n for _ in range(n)]
            m2 = [[Decimal(0)] * n for _ in range(n)]
            for i in range(n):
                m2[i][i] += Decimal(d0.numerator) / Decimal(d0.denominator) / (h * h)
                for k in range(1, self.r + 1):
                    ck = Decimal(c[k - 1].numerator) / Decimal(c[k - 1].denominator) / h
                    dk = Decimal(d[k - 1].numerator) / Decimal(d[k - 1].denominator) / (h * h)
                    m1[i][(i + k) % n] += ck
                    m1[i][(i - k) % n] -= ck
                    m2[i][(i + k) % n] += dk
                    m2[i][(i - k) % n] += dk
            self.D1.append(m1)
            self.D2.append(m2)

    def idx(self, x, y, z):
        nx, ny, _ = self.n
        return (z * ny + y) * nx + x

    def apply(self, M, f, axis):
        nx, ny, nz = self.n
        out = [Decimal(0)] * len(f)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    pos = (x, y, z)
                    row = M[pos[axis]]
                    s = Decimal(0)
                    for j, w in enumerate(row):
                        if w == 0:
                            continue
                        q = list(pos)
                        q[axis] = j
                        s += w * f[self.idx(*q)]
                    out[self.idx(x, y, z)] = s
        return out

    def d1(self, f, axis):
        return self.apply(self.D1[axis], f, axis)

    def d2(self, f, axis):
        return self.apply(self.D2[axis], f, axis)


def _to_dec(a):
    return [Decimal(float(v)) for v in a]


def residual(box: Box, Q, Re, Mach, gamma, Pr, visc_form=0):
    """Q: list of 5 flat lists of Decimal.  Returns 5 flat lists of Decimal."""
    Re, Mach, gamma, Pr = (Decimal(float(v)) for v in (Re, Mach, gamma, Pr))
    npt = len(Q[0])
    half = Decimal(1) / 2
    rho = Q[0]
    u = [[Q[1 + i][p] / rho[p] for p in range(npt)] for i in range(3)]
    ke = [half * rho[p] * sum(u[i][p] * u[i][p] for i in range(3)) for p in range(npt)]
    pr = [(gamma - 1) * (Q[4][p] - ke[p]) for p in range(npt)]
    T = [gamma * Mach * Mach * pr[p] / rho[p] for p in range(npt)]
    kappa = 1 / ((gamma - 1) * Mach * Mach * Pr * Re)
    # gradient: Gr[i][j] = D_j u_i
    Gr = [[box.d1(u[i], j) for j in range(3)] for i in range(3)]
    div = [Gr[0][0][p] + Gr[1][1][p] + Gr[2][2][p] for p in range(npt)]

    R = [[Decimal(0)] * npt for _ in range(5)]
    # convective (skew-symmetric) terms
    for m in range(5):
        a = Q[m]
        for j in range(3):
            flux = box.d1([a[p] * u[j][p] for p in range(npt)], j)
            da = box.d1(a, j)
            for p in range(npt):
                R[m][p] -= half * (flux[p] + u[j][p] * da[p] + a[p] * Gr[j][j][p])
    # pressure
    for i in range(3):
        dp = box.d1(pr, i)
        for p in range(npt):
            R[1 + i][p] -= dp[p]
    for j in range(3):
        dpu = box.d1([u[j][p] * pr[p] for p in range(npt)], j)
        for p in range(npt):
            R[4][p] -= dpu[p]
    # viscous momentum, simplified algebra
    L = [[box.d2(u[i], j) for j in range(3)] for i in range(3)]  # L[i][j] = L_j u_i
    dtau = []
    third = Decimal(1) / 3
    for i in range(3):
        cross = [Decimal(0)] * npt
        for k in range(3):
            if k != i:
                dk = box.d1(Gr[k][k], i)  # D_i (D_k u_k)
                cross = [cross[p] + dk[p] for p in range(npt)]
        v = [(L[i][0][p] + L[i][1][p] + L[i][2][p] + third * (L[i][i][p] + cross[p])) / Re
             for p in range(npt)]
        dtau.append(v)
        for p in range(npt):
            R[1 + i][p] += v[p]
    # heat flux
    for j in range(3):
        lt = box.d2(T, j)
        for p in range(npt):
            R[4][p] += kappa * lt[p]
    # viscous work
    two_thirds = Decimal(2) / 3

    def tau(i, j, p):
        t = Gr[i][j][p] + Gr[j][i][p]
        if i == j:
            t -= two_thirds * div[p]
        return t / Re

    if visc_form == 0:
        for j in range(3):
            w = [sum(u[i][p] * tau(i, j, p) for i in range(3)) for p in range(npt)]
            dw = box.d1(w, j)
            for p in range(npt):
                R[4][p] += dw[p]
    else:
        for p in range(npt):
            R[4][p] += sum(u[i][p] * dtau[i][p] for i in range(3))
            R[4][p] += sum(tau(i, j, p) * Gr[i][j][p] for i in range(3) for j in range(3))
    return R


RK_ALPHA = (Fraction(2, 3), Fraction(5, 12), Fraction(3, 5))
RK_BETA = (Fraction(1, 4), Fraction(3, 20), Fraction(3, 5))


def rk3(box: Box, Q, nsteps, dt, Re, Mach, gamma, Pr, visc_form=0):
    """Low-storage RK3 on Decimal lists; dt is taken as the exact binary64 value."""
    dt = Decimal(float(dt))
    U = [list(f) for f in Q]
    for _ in range(nsteps):
        q = [list(f) for f in U]
        for k in range(3):
            R = residual(box, q, Re, Mach, gamma, Pr, visc_form)
            a = Decimal(RK_ALPHA[k].numerator) / RK_ALPHA[k].denominator * dt
            b = Decimal(RK_BETA[k].numerator) / RK_BETA[k].denominator * dt
            q = [[U[m][p] + a * R[m][p] for p in range(len(U[m]))] for m in range(5)]
            U = [[U[m][p] + b * R[m][p] for p in range(len(U[m]))] for m in range(5)]
    return U


def from_numpy(Q):
    return [_to_dec(Q[m].ravel()) for m in range(5)]


def to_float(Qd):
    import numpy as np
    return np.array([[float(v) for v in f] for f in Qd])

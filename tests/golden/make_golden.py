"""Writes tgv_enstrophy0.json: the discrete enstrophy of the Taylor-Green
initial state, from its closed form kappa1^2 (3/8 - 5 gamma M^2 / 128).

kappa1 = (2/h) sum_k c_k sin(k h) is the modified wavenumber of mode 1 for the
order-2r central first derivative (weights from exact Taylor matching in
rationals).  Derivation: with a = cos 2x, b = cos 2y, c = cos 2z the discrete
vorticity of the initial velocity is kappa1 * (-cos x sin y sin z,
-sin x cos y sin z, 2 sin x sin y cos z) and rho = 1 + gamma M^2 (a+b)(2+c)/16,
so <rho |omega|^2 / 2> = kappa1^2 [3/8 + (gamma M^2/32) <(a+b)(2+c) W>] with
<(a+b)(2+c) W> = -5/4 whenever the grid averages of a, a^2 equal their
continuous values (N not in {1, 2, 4}).  No solver code is called.
"""
import json
import math
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from tests.bruteforce import first_derivative_weights  # noqa: E402

GAMMA, MACH = 1.4, 0.1


def enstrophy0(n, order):
    h = 2 * math.pi / n
    c = first_derivative_weights(order // 2)
    k1 = 2 * sum(float(ck) * math.sin((k + 1) * h) for k, ck in enumerate(c)) / h
    gM2 = GAMMA * MACH ** 2
    return k1 * k1 * (3 / 8 - 5 * gM2 / 128)


if __name__ == "__main__":
    cases = [dict(n=n, order=o, enstrophy0=enstrophy0(n, o))
             for n, o in ((8, 4), (32, 4), (64, 4), (32, 8), (16, 2), (48, 6))]
    out = {"_source": "closed form, written by tests/golden/make_golden.py (no solver code)",
           "gamma": GAMMA, "Mach": MACH, "continuous_limit": 3 / 8 - 5 * GAMMA * MACH ** 2 / 128,
           "cases": cases}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tgv_enstrophy0.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")

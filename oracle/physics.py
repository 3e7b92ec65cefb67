"""Phase mobilities and fractional flow.

Eq. brooksCorey: lambda_w = k_rw(s)/eta_w, lambda_o = k_ro(s)/eta_o,
lambda = lambda_w + lambda_o. The paper's runs use linear relative
permeabilities k_rw = s, k_ro = 1 - s (Section 6); the quadratic Corey law
k_rw = s^2, k_ro = (1 - s)^2 is the other supported law.
Eq. frationalFlow: f_w = lambda_w / (lambda_w + lambda_o).
"""
from __future__ import annotations

import numpy as np


def relperm(s, law: str):
    s = np.asarray(s, dtype=np.float64)
    if law == "corey":
        return s * s, (1.0 - s) * (1.0 - s)
    if law == "linear":
        return s, 1.0 - s
    raise ValueError(law)


def mobilities(s, eta_w: float, eta_o: float, law: str):
    krw, kro = relperm(s, law)
    lw = krw / eta_w
    lo = kro / eta_o
    return lw, lo, lw + lo


def total_mobility(s, eta_w, eta_o, law):
    return mobilities(s, eta_w, eta_o, law)[2]


def frac_flow(s, eta_w, eta_o, law):
    lw, lo, lt = mobilities(s, eta_w, eta_o, law)
    return lw / lt


def max_frac_flow_slope(eta_w: float, eta_o: float, law: str) -> float:
    """L_f = max over [0, 1] of f_w'(s), used by the CFL time step.

    The derivative is evaluated by central differences on a 1e5-point sample,
    then refined by golden-section search around the best sample."""
    def dfw(s):
        h = 1e-7
        a = np.clip(s - h, 0.0, 1.0)
        b = np.clip(s + h, 0.0, 1.0)
        return (frac_flow(b, eta_w, eta_o, law) - frac_flow(a, eta_w, eta_o, law)) / (b - a)

    xs = np.linspace(0.0, 1.0, 100001)
    d = dfw(xs)
    k = int(np.argmax(d))
    lo = xs[max(k - 1, 0)]
    hi = xs[min(k + 1, len(xs) - 1)]
    gr = (np.sqrt(5.0) - 1.0) / 2.0
    for _ in range(80):
        c = hi - gr * (hi - lo)
        e = lo + gr * (hi - lo)
        if dfw(c) > dfw(e):
            hi = e
        else:
            lo = c
    return float(max(d[k], dfw(0.5 * (lo + hi))))

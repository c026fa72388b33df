"""Oracle side of the temporal profiles (TEST INFRASTRUCTURE ONLY).

f(t) is written out piecewise as the paper defines it (Section 3, "General
diffusion-encoding sequence", cos-OGSE with w = 2 pi n / delta and
tau = (delta + Delta)/2; the other profiles of Section 4 built the same way),
and everything else is obtained by adaptive numerical integration (SciPy
`quad`), a different route from the library's closed forms:
  F_n   = sum over steps of int_{t_{k-1}}^{t_k} f,
  int F^2 = int_0^TE (int_0^t f)^2 dt   (nested quadrature).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def f_of_t(kind, s, delta, Delta, n_periods=1, ramp=None):
    """The profile f(s) itself (scalar s)."""
    if kind == "pgse":
        if 0.0 <= s <= delta:
            return 1.0
        if Delta < s <= Delta + delta:
            return -1.0
        return 0.0
    if kind == "double_pgse":
        T1 = Delta + delta
        return f_of_t("pgse", s, delta, Delta) + (f_of_t("pgse", s - T1, delta, Delta) if s > T1 else 0.0)
    if kind in ("cos_ogse", "sin_ogse"):
        w = 2.0 * math.pi * n_periods / delta
        tau = 0.5 * (delta + Delta)
        g = math.cos if kind == "cos_ogse" else math.sin
        if 0.0 <= s <= delta:
            return g(w * s)
        if tau < s <= tau + delta:
            return -g(w * (s - tau))
        return 0.0
    if kind in ("trapezoid", "double_trapezoid"):
        r = ramp if ramp is not None else delta / 10.0

        def lobe(x):  # one trapezoid on [0, delta]
            if x < 0.0 or x > delta:
                return 0.0
            if x < r:
                return x / r
            if x > delta - r:
                return (delta - x) / r
            return 1.0

        val = lobe(s) - lobe(s - Delta)
        if kind == "double_trapezoid":
            T1 = Delta + delta
            val += lobe(s - T1) - lobe(s - T1 - Delta)
        return val
    raise ValueError(kind)


def _points(kind, delta, Delta, n_periods, ramp):
    r = (ramp if ramp is not None else delta / 10.0)
    tau = 0.5 * (delta + Delta)
    T1 = Delta + delta
    pts = [0.0, delta, Delta, Delta + delta, tau, tau + delta, T1, T1 + delta, T1 + Delta, T1 + Delta + delta]
    pts += [r, delta - r, Delta + r, Delta + delta - r, T1 + r, T1 + delta - r, T1 + Delta + r,
            T1 + Delta + delta - r]
    return sorted(set(pts))


def _integral_f(kind, a, b, delta, Delta, n_periods, ramp):
    if b <= a:
        return 0.0
    pts = [p for p in _points(kind, delta, Delta, n_periods, ramp) if a < p < b]
    val, _ = integrate.quad(lambda s: f_of_t(kind, s, delta, Delta, n_periods, ramp), a, b, points=pts or None,
                            epsabs=1e-13, epsrel=1e-13, limit=200)
    return val


def tables(kind, delta, Delta, TE, dt, n_periods=1, ramp=None):
    """(f_bar[n_steps], F[n_steps + 1], int_0^TE F^2)."""
    n = int(round(TE / dt))
    steps = np.array([_integral_f(kind, (k - 1) * dt, k * dt, delta, Delta, n_periods, ramp)
                      for k in range(1, n + 1)])
    F = np.concatenate([[0.0], np.cumsum(steps)])
    fbar = steps / dt

    def F_at(t):
        k = int(t // dt)
        k = min(k, n)
        return F[k] + _integral_f(kind, k * dt, t, delta, Delta, n_periods, ramp)

    pts = [p for p in _points(kind, delta, Delta, n_periods, ramp) if 0.0 < p < TE]
    I, _ = integrate.quad(lambda t: F_at(t) ** 2, 0.0, TE, points=pts or None, epsabs=1e-10, epsrel=1e-12,
                          limit=400)
    return fbar, F, I

"""Temporal profiles f(t) of the diffusion-encoding gradient, as the tables
`bt_set_profile` takes: F(t_n) = int_0^{t_n} f on the time grid and
int_0^TE F^2 (for b = q^2 int F^2, Eq. b_value).

The paper's framework accepts arbitrary profiles (Section 3, "General
diffusion-encoding sequence") and shows PGSE, double PGSE, cos-OGSE, sin-OGSE,
trapezoidal and double trapezoidal PGSE (Section 4).  Here F is written in
closed form per profile and int F^2 is integrated with composite
Gauss-Legendre quadrature between the profile's breakpoints (F is smooth
between them).  Times in us.

Profiles (delta = lobe length, Delta as below):
  pgse              f = +1 on [0, delta], -1 on [Delta, Delta + delta]
  double_pgse       two PGSE blocks, the second starting at Delta + delta
  cos_ogse          f = cos(w s) on [0, delta], -cos(w (s - tau)) on (tau, tau + delta],
                    w = 2 pi n / delta, tau = (delta + Delta) / 2 (the paper's definition)
  sin_ogse          as cos_ogse with sin
  trapezoid         PGSE lobes with linear ramps of length `ramp` at both ends
  double_trapezoid  two trapezoid blocks, the second starting at Delta + delta
"""
from __future__ import annotations

import math

import numpy as np

KINDS = ("pgse", "double_pgse", "cos_ogse", "sin_ogse", "trapezoid", "double_trapezoid")


def _clamp(x, lo, hi):
    return np.minimum(np.maximum(x, lo), hi)


def _lobe_pgse(x, delta):
    return _clamp(x, 0.0, delta)


def _lobe_trap(x, delta, ramp):
    """int_0^x of the trapezoid lobe (0 -> 1 over ramp, flat, 1 -> 0 over ramp)."""
    x = _clamp(x, 0.0, delta)
    a = x * x / (2.0 * ramp)
    b = ramp / 2.0 + (x - ramp)
    c = delta - ramp - (delta - x) ** 2 / (2.0 * ramp)
    return np.where(x <= ramp, a, np.where(x <= delta - ramp, b, c))


def F_of_t(kind, t, delta, Delta, n_periods=1, ramp=None):
    """F(t) = int_0^t f(s) ds, vectorised over t."""
    t = np.asarray(t, dtype=np.float64)
    if kind == "pgse":
        return _lobe_pgse(t, delta) - _lobe_pgse(t - Delta, delta)
    if kind == "double_pgse":
        T1 = Delta + delta
        return F_of_t("pgse", t, delta, Delta) + F_of_t("pgse", np.maximum(t - T1, 0.0), delta, Delta)
    if kind in ("cos_ogse", "sin_ogse"):
        w = 2.0 * math.pi * n_periods / delta
        tau = 0.5 * (delta + Delta)
        if kind == "cos_ogse":
            S = lambda x: np.sin(w * x) / w
        else:
            S = lambda x: (1.0 - np.cos(w * x)) / w
        return S(_clamp(t, 0.0, delta)) - S(_clamp(t - tau, 0.0, delta))
    if kind in ("trapezoid", "double_trapezoid"):
        r = ramp if ramp is not None else delta / 10.0
        single = _lobe_trap(t, delta, r) - _lobe_trap(t - Delta, delta, r)
        if kind == "trapezoid":
            return single
        T1 = Delta + delta
        return single + F_of_t("trapezoid", np.maximum(t - T1, 0.0), delta, Delta, ramp=r)
    raise ValueError(f"unknown profile {kind!r}")


def breakpoints(kind, delta, Delta, TE, n_periods=1, ramp=None):
    """Times where f (hence F') is not smooth, within [0, TE]."""
    pts = [0.0, TE]
    if kind in ("pgse", "double_pgse", "trapezoid", "double_trapezoid"):
        r = (ramp if ramp is not None else delta / 10.0) if "trap" in kind else 0.0
        starts = [0.0, Delta]
        if kind.startswith("double"):
            starts += [Delta + delta, 2 * Delta + delta]
        for s0 in starts:
            pts += [s0, s0 + r, s0 + delta - r, s0 + delta]
    else:
        tau = 0.5 * (delta + Delta)
        pts += [0.0, delta, tau, tau + delta]
    return sorted({p for p in pts if 0.0 <= p <= TE})


def int_F2(kind, delta, Delta, TE, n_periods=1, ramp=None, pieces=64, order=10):
    """int_0^TE F(t)^2 dt by composite Gauss-Legendre between breakpoints."""
    xg, wg = np.polynomial.legendre.leggauss(order)
    bp = breakpoints(kind, delta, Delta, TE, n_periods, ramp)
    total = 0.0
    for a, b in zip(bp[:-1], bp[1:]):
        if b <= a:
            continue
        edges = np.linspace(a, b, pieces + 1)
        for lo, hi in zip(edges[:-1], edges[1:]):
            t = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
            total += 0.5 * (hi - lo) * float(np.dot(wg, F_of_t(kind, t, delta, Delta, n_periods, ramp) ** 2))
    return total


def tables(kind, delta, Delta, TE, dt, n_periods=1, ramp=None):
    """(F[n_steps + 1], int_0^TE F^2) for bt_set_profile; TE must be a multiple of dt."""
    if kind not in KINDS:
        raise ValueError(f"unknown profile {kind!r}")
    n = int(round(TE / dt))
    if n < 1 or abs(n * dt - TE) > 1e-9 * TE:
        raise ValueError("TE must be a positive multiple of dt")
    F = F_of_t(kind, np.arange(n + 1) * dt, delta, Delta, n_periods, ramp)
    F[0] = 0.0
    return F, int_F2(kind, delta, Delta, TE, n_periods, ramp)

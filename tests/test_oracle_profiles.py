"""Pins of the arbitrary temporal profiles (Section 3, "General
diffusion-encoding sequence"; the profiles of Section 4).  The oracle
integrates f numerically; these tests fix it against closed forms of
int_0^TE F^2 derived by hand, against the library's independent closed-form
tables (bt_waveform_tables through the C ABI, host code, no GPU), and through
the exact free-diffusion solution of the periodic box, whose continuum limit
is exp(-b D) with b = q^2 int F^2 (Eq. b_value)."""
import math

import numpy as np
import pytest

import geom
import oracle
from oracle import btoracle as bo
from oracle import profiles as op
from paper_1908_01719_gb300 import bt

DELTA, BIG_DELTA, DT = 2000.0, 3000.0, 50.0


def _te(kind, delta=DELTA, Delta=BIG_DELTA):
    if kind in ("cos_ogse", "sin_ogse"):
        return 0.5 * (delta + Delta) + delta
    if kind.startswith("double"):
        return 2 * (Delta + delta)
    return Delta + delta


@pytest.mark.parametrize("kind,n,closed", [
    ("pgse", 1, lambda d, D, w: d * d * (D - d / 3.0)),
    ("double_pgse", 1, lambda d, D, w: 2 * d * d * (D - d / 3.0)),
    ("cos_ogse", 2, lambda d, D, w: d / w ** 2),
    ("sin_ogse", 2, lambda d, D, w: 3 * d / w ** 2),
    ("cos_ogse", 3, lambda d, D, w: d / w ** 2),
])
def test_oracle_int_F2_closed_forms(kind, n, closed):
    """int F^2: PGSE delta^2 (Delta - delta/3); two PGSE blocks twice that;
    cos-OGSE with n whole periods: F = sin(w t)/w on each lobe, int = delta/w^2;
    sin-OGSE: F = (1 - cos(w t))/w, int = 3 delta / w^2."""
    w = 2 * math.pi * n / DELTA
    TE = _te(kind)
    fbar, F, I = op.tables(kind, DELTA, BIG_DELTA, TE, DT, n_periods=n)
    assert abs(I - closed(DELTA, BIG_DELTA, w)) <= 1e-9 * closed(DELTA, BIG_DELTA, w)
    assert abs(F[-1]) < 1e-9 * DELTA            # balanced: F(TE) = 0
    assert np.allclose(np.diff(F) / DT, fbar, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind", ["pgse", "double_pgse", "cos_ogse", "sin_ogse", "trapezoid", "double_trapezoid"])
def test_library_tables_match_oracle(kind):
    """Closed-form F and Gauss-Legendre int F^2 (library) against adaptive
    quadrature of f (oracle): two independent routes."""
    TE = _te(kind)
    _, Fo, Io = op.tables(kind, DELTA, BIG_DELTA, TE, DT, n_periods=2, ramp=150.0)
    Fl, Il = bt.bt_waveform_tables(kind, DELTA, BIG_DELTA, TE, DT, n_periods=2, ramp=150.0)
    assert np.max(np.abs(Fl - Fo)) < 1e-9 * DELTA
    assert abs(Il - Io) < 1e-10 * Io


def test_library_refuses_invalid_profiles():
    """The library's profile parameters are checked before any table is made."""
    TE = _te("pgse")
    for args in [("pgse", 0.0, BIG_DELTA, TE, DT), ("pgse", DELTA, DELTA / 2, TE, DT),
                 ("pgse", DELTA, BIG_DELTA, TE + 1.0, DT), ("pgse", DELTA, BIG_DELTA, DELTA, DT),
                 ("cos_ogse", DELTA, BIG_DELTA, _te("cos_ogse"), DT, 0),
                 ("trapezoid", DELTA, BIG_DELTA, TE, DT, 1, 0.6 * DELTA)]:
        with pytest.raises(bt.BtError):
            bt.bt_waveform_tables(*args)
    F, I = bt.bt_waveform_tables("pgse", DELTA, BIG_DELTA, TE, DT)
    assert len(F) == int(round(TE / DT)) + 1 and F[0] == 0.0


def test_trapezoid_tends_to_pgse():
    """A ramp of zero length is the PGSE; int F^2 moves smoothly to its value."""
    TE = _te("trapezoid")
    pg = DELTA ** 2 * (BIG_DELTA - DELTA / 3.0)
    errs = [abs(op.tables("trapezoid", DELTA, BIG_DELTA, TE, DT, ramp=r)[2] - pg) / pg for r in (200.0, 100.0, 50.0)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.05
    assert 1.7 < errs[0] / errs[1] < 2.3      # first order in the ramp length


@pytest.mark.parametrize("kind", ["cos_ogse", "double_pgse"])
def test_free_periodic_box_exact_and_limit(kind):
    """Periodic box, no compartments, transformed frame: u stays spatially
    constant and S/|Omega| = prod_n (1 - (1-th) dt D q^2 F_{n-1}^2) /
    (1 + th dt D q^2 F_n^2) exactly, with the profile's own F; as dt -> 0 this
    tends to exp(-b D), second order in dt."""
    D, b = 2e-3, 800.0
    errs = []
    for dt in (50.0, 25.0):
        p = geom.free_periodic_box(n=3, L=6.0, dt=dt, D=D, bvals=(b,))
        p.delta, p.Delta = DELTA, BIG_DELTA
        p.TE = _te(kind)
        p.profile = {"kind": kind, "n_periods": 2}
        S = bo.run(p)[0] / 216.0
        _, F, I = op.tables(kind, p.delta, p.Delta, p.TE, dt, n_periods=2)
        q2 = b / I
        prod = np.prod((1 - 0.5 * dt * D * q2 * F[:-1] ** 2) / (1 + 0.5 * dt * D * q2 * F[1:] ** 2))
        assert abs(S - prod) < 1e-12
        errs.append(abs(S.real - math.exp(-b * D)))
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_ogse_decays_faster_in_a_disk():
    """Section 4's comparison of six profiles in a disk of radius 5 um with
    delta = Delta = 10 ms: at equal b the OGSE signals decay faster than the
    PGSE, double PGSE and trapezoidal ones (shorter effective diffusion time,
    less restriction)."""
    TE = {"pgse": 20000.0, "double_pgse": 40000.0, "cos_ogse": 20000.0, "sin_ogse": 20000.0,
          "trapezoid": 20000.0, "double_trapezoid": 40000.0}
    S = {}
    for kind, te in TE.items():
        p = geom.polar_disk(8, dt=100.0, bvals=(1000.0, 3000.0))
        p.delta, p.Delta, p.TE = 10000.0, 10000.0, te
        p.profile = {"kind": kind, "n_periods": 1, "ramp": 1000.0}
        S[kind] = oracle.run(p).real
    for og in ("cos_ogse", "sin_ogse"):
        for other in ("pgse", "double_pgse", "trapezoid", "double_trapezoid"):
            assert np.all(S[og] < S[other]), (og, other, S[og], S[other])

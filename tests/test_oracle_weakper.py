"""Pins of the weak pseudo-periodic conditions (Appendix B, artificial
permeability on the faces of a box meshed without periodicity).

- g = 0: the coupling of partner faces cancels the boundary mass on a
  constant field (C 1 = B 1 for a matching mesh), so S(t_n) = |Omega| exactly.
- Reversing the gradient conjugates the signal (every phase flips sign).
- The partner side is taken from the previous step: the scheme is first
  order in dt (successive differences halve when dt halves).
- With kappa_e ten times the default D/h and dt = 12.5 us the free-diffusion
  signal is within 0.03 of exp(-b D), the pseudo-periodic value, as Appendix
  B's comparison shows the method approaching the strong conditions."""
import math

import numpy as np

import geom
import oracle


def _box(dt=50.0, b=1000.0, dirs=((1.0, 0.0, 0.0),), kappa_e=None, n=6):
    p = geom.free_periodic_box(n=n, L=8.0, dt=dt, bvals=(b,), dirs=dirs)
    p.periodic_mask = 0
    p.transformed = False
    p.weak_periodic = {"axes": 7, "kappa_e": kappa_e}
    return p


def test_constant_field_conserved_at_zero_gradient():
    p = _box(b=0.0)
    S, H = oracle.run(p, return_history=True)
    assert np.max(np.abs(H[0] - 512.0)) < 1e-11 * 512.0


def test_reversed_gradient_conjugates_signal():
    d = (0.3, 0.4, math.sqrt(0.75))
    a = oracle.run(_box(dirs=(d,), n=4))[0]
    b = oracle.run(_box(dirs=(tuple(-x for x in d),), n=4))[0]
    assert abs(a - np.conj(b)) < 1e-12 * abs(a)


def test_first_order_in_dt():
    S = [oracle.run(_box(dt=dt, kappa_e=1.5e-2, n=4))[0] for dt in (50.0, 25.0, 12.5)]
    d1, d2 = abs(S[0] - S[1]), abs(S[1] - S[2])
    assert 1.6 < d1 / d2 < 2.4


def test_approaches_pseudo_periodic_value():
    S = oracle.run(_box(dt=12.5, kappa_e=1.5e-2))[0] / 512.0
    assert abs(S - math.exp(-1000.0 * 2e-3)) < 0.03


# ---------------------------------------------------------------- 2-D (boundary edges)
def _square(dt=50.0, b=1000.0, dirs=((1.0, 0.0, 0.0),), kappa_e=None, n=8):
    p = geom.free_periodic_square(n=n, L=8.0, dt=dt, bvals=(b,), dirs=dirs)
    p.periodic_mask = 0
    p.transformed = False
    p.weak_periodic = {"axes": 3, "kappa_e": kappa_e}
    return p


def test_square_constant_field_conserved_at_zero_gradient():
    S, H = oracle.run(_square(b=0.0), return_history=True)
    assert np.max(np.abs(H[0] - 64.0)) < 1e-11 * 64.0


def test_square_reversed_gradient_conjugates_and_first_order():
    d = (0.6, 0.8, 0.0)
    a = oracle.run(_square(dirs=(d,), n=4, b=2500.0))[0]
    b = oracle.run(_square(dirs=(tuple(-x for x in d),), n=4, b=2500.0))[0]
    assert abs(a - np.conj(b)) < 1e-12 * abs(a)
    S = [oracle.run(_square(dt=dt, kappa_e=1.5e-2, n=4))[0] for dt in (50.0, 25.0, 12.5)]
    d1, d2 = abs(S[0] - S[1]), abs(S[1] - S[2])
    assert 1.6 < d1 / d2 < 2.4


def test_square_approaches_pseudo_periodic_value():
    S = oracle.run(_square(dt=12.5, kappa_e=1.5e-2))[0] / 64.0
    assert abs(S - math.exp(-1000.0 * 2e-3)) < 0.03


def test_square_with_disk_weak_approaches_strong_conditions():
    """The paper's 2-D comparison of the two routes (Appendix B): a disk in a
    square, gradient along (1, 1)/sqrt(2), delta 10 ms, Delta 13 ms.  The
    strong route meshes the square periodically (transformed frame); the weak
    route couples the sides of the same, non-periodic mesh.  The gap shrinks
    as dt is halved (the partner term lags one step)."""
    d = (1 / math.sqrt(2), 1 / math.sqrt(2), 0.0)

    def make(dt, strong):
        p = geom.square_disk(n=16, L=10.0, R=3.0, dt=dt, kappa=1e-4, bvals=(1000.0,), dirs=(d,))
        p.delta, p.Delta, p.TE = 10000.0, 13000.0, 23000.0
        if strong:
            p.periodic_mask, p.transformed = 3, True
        else:
            p.weak_periodic = {"axes": 3, "kappa_e": 1e-2}
        return p
    gaps = []
    for dt in (50.0, 25.0, 12.5):
        Ss, Sw = oracle.run(make(dt, True))[0], oracle.run(make(dt, False))[0]
        gaps.append(abs(Sw - Ss) / abs(Ss))
    assert gaps[0] > gaps[1] > gaps[2] and gaps[2] < 0.08, gaps


# ---------------------------------------------------------------- non-matching sides (projection)
def _sheared(eps, dt=50.0, b=1000.0, dirs=((1.0, 0.0, 0.0),), kappa_e=None, n=4):
    p = geom.sheared_box(n=n, L=8.0, eps=eps, dt=dt, bvals=(b,), dirs=dirs)
    p.weak_periodic = {"axes": 7, "kappa_e": kappa_e}
    return p


def test_projection_reproduces_constants_on_non_matching_sides():
    """With the x sides sheared against each other, the projected coupling
    still satisfies C 1 = B 1 (interpolation reproduces constants), so the
    signal stays |Omega| at g = 0."""
    from oracle import btoracle as bo
    from oracle import weakper
    p = _sheared(0.3, b=0.0, n=6)
    a = bo.assemble(p)
    B, pairs, ke, L = weakper.operators(p, a, 7)
    C = weakper.coupling(pairs, a["n"], 0.0, (1.0, 0.0, 0.0), L, 0.0)
    one = np.ones(a["n"])
    assert np.max(np.abs(C @ one - B @ one)) < 1e-13 * np.max(np.abs(B @ one))
    S, H = oracle.run(p, return_history=True)
    assert np.max(np.abs(H[0] - 512.0)) < 1e-11 * 512.0


def test_projection_conjugates_and_tends_to_the_matching_solution():
    d = (0.3, 0.4, math.sqrt(0.75))
    a = oracle.run(_sheared(0.3, dirs=(d,)))[0]
    b = oracle.run(_sheared(0.3, dirs=(tuple(-x for x in d),)))[0]
    assert abs(a - np.conj(b)) < 1e-12 * abs(a)
    S0 = oracle.run(_sheared(0.0))[0]
    gaps = [abs(oracle.run(_sheared(e))[0] - S0) for e in (0.4, 0.2, 0.1)]
    assert gaps[0] > gaps[1] > gaps[2] and gaps[2] < 0.01 * abs(S0), gaps


def test_projection_approaches_pseudo_periodic_value():
    S = oracle.run(_sheared(0.3, dt=12.5, kappa_e=1.5e-2, n=6))[0] / 512.0
    assert abs(S - math.exp(-1000.0 * 2e-3)) < 0.03

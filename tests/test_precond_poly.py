"""The fixed Chebyshev polynomial preconditioner (library host code, no GPU):
the baseline the learned polynomial is compared with.  Pinned against numpy's
Chebyshev series (Clenshaw evaluation in the Chebyshev basis, independent of
the library's monomial expansion), the minimax property of T_9 and the
closed form of the loss on a diagonal operator."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npc

from paper_1908_01719_gb300 import bt


def residual(c, lam):
    """1 - lam p(lam) with p = sum_j c_j lam^j."""
    return 1.0 - lam * np.polyval(c[::-1], lam)


@pytest.mark.parametrize("lo,hi", [(0.05, 2.5), (0.3, 1.7), (1e-3, 4.0)])
def test_chebyshev_residual_polynomial(lo, hi):
    c = bt.bt_chebyshev_poly(lo, hi)
    lam = np.linspace(0.0, 1.2 * hi, 2001)
    t9 = np.zeros(10)
    t9[9] = 1.0
    x = lambda l: (hi + lo - 2.0 * l) / (hi - lo)
    ref = npc.chebval(x(lam), t9) / npc.chebval(x(0.0), t9)
    assert np.max(np.abs(residual(c, lam) - ref)) < 1e-9 * max(1.0, np.max(np.abs(ref)))
    assert abs(residual(c, 0.0) - 1.0) < 1e-15


def test_chebyshev_minimax_equioscillation():
    """On [lo, hi] the residual reaches +-1/T_9(a) at the ten extrema of T_9
    with alternating signs and never exceeds it."""
    lo, hi = 0.1, 2.0
    c = bt.bt_chebyshev_poly(lo, hi)
    a = (hi + lo) / (hi - lo)
    eps = 1.0 / np.cosh(9 * np.arccosh(a))
    ext = 0.5 * (hi + lo) - 0.5 * (hi - lo) * np.cos(np.pi * np.arange(10) / 9)  # x = cos(k pi / 9)
    r = residual(c, ext)
    assert np.allclose(np.abs(r), eps, rtol=1e-8)
    assert np.all(np.sign(r[1:]) == -np.sign(r[:-1]))
    lam = np.linspace(lo, hi, 5001)
    assert np.max(np.abs(residual(c, lam))) <= eps * (1 + 1e-8)


def test_chebyshev_refuses_bad_intervals():
    for lo, hi in [(0.0, 1.0), (1.0, 1.0), (2.0, 1.0), (0.1, np.inf)]:
        with pytest.raises(bt.BtError):
            bt.bt_chebyshev_poly(lo, hi)


def spectral_samples(lam, w):
    """Samples of a diagonal operator B = diag(lam) with D = I and residual
    weights w: y_j = lam^(j+1) r, so G_jk = sum w lam^(j+k+2), h_j = sum w lam^(j+1)."""
    P = lam[None, :] ** (np.arange(9)[:, None] + 1)  # [9][m]
    G = (P * w) @ P.T
    h = P @ w
    return G[None], h[None]


def test_fit_on_a_diagonal_operator():
    """For a spectrum spread over [0.2, 2.5] the fitted interval does at least
    as well as the true interval, the loss it reports is sum w (1 - l p(l))^2,
    and it beats Jacobi (c = e_0, loss sum w (1 - l)^2)."""
    rng = np.random.default_rng(3)
    lam = np.sort(rng.uniform(0.2, 2.5, 400))
    w = rng.uniform(0.5, 1.5, 400)
    w /= w.sum()
    G, h = spectral_samples(lam, w)
    lo, hi, c, loss = bt.bt_fit_chebyshev(G, h, rel_err=1e-14)
    # the monomial form 1 - 2 c.h + c.G c cancels: allow its rounding bound
    mag = 1.0 + 2 * np.abs(c) @ np.abs(h[0]) + np.abs(c) @ np.abs(G[0]) @ np.abs(c)
    assert abs(loss - np.sum(w * residual(c, lam) ** 2)) < 64 * np.finfo(float).eps * mag
    true = np.sum(w * residual(bt.bt_chebyshev_poly(0.2, 2.5), lam) ** 2)
    assert loss <= true * 1.001
    assert loss < 0.05 * np.sum(w * (1.0 - lam) ** 2)
    assert 0.05 < lo < 0.4 and 2.0 < hi < 3.0


def test_fit_covers_the_estimated_spectrum():
    """Residuals made mostly of low modes: the loss alone would prefer an
    interval that stops short of the top eigenvalues; the fit keeps hi at or
    above 1.05 |y_8|/|y_7| (a power-iteration estimate of the top modulus),
    so the residual polynomial stays at most 1 in modulus over the spectrum."""
    lam = np.linspace(0.3, 3.0, 300)
    w = np.exp(-4.0 * lam)
    w /= w.sum()
    G, h = spectral_samples(lam, w)
    est = np.sqrt(G[0, 8, 8] / G[0, 7, 7])
    lo, hi, c, loss = bt.bt_fit_chebyshev(G, h, rel_err=1e-14)
    assert hi >= 1.05 * est * (1 - 1e-12) and est <= lam.max()
    assert np.max(np.abs(residual(c, lam[lam <= hi]))) <= 1.0 + 1e-9


def test_fit_on_noisy_data_is_not_fooled():
    """G and h perturbed at relative 1e-6 (the collected data's FP32 Krylov
    vectors): with that accuracy declared, the fitted polynomial's true loss
    (exact data) stays close to the exact-data fit and the reported loss is
    positive; declaring exact data instead lets rounding pass for progress."""
    rng = np.random.default_rng(5)
    lam = np.sort(rng.uniform(0.02, 2.5, 400))
    w = rng.uniform(0.5, 1.5, 400)
    w /= w.sum()
    G, h = spectral_samples(lam, w)
    Gn = G * (1 + 1e-6 * rng.standard_normal(G.shape))
    Gn = 0.5 * (Gn + Gn.transpose(0, 2, 1))
    hn = h * (1 + 1e-6 * rng.standard_normal(h.shape))
    true = lambda c: np.sum(w * residual(c, lam) ** 2)
    _, _, c_exact, _ = bt.bt_fit_chebyshev(G, h, rel_err=1e-14)
    lo, hi, c, loss = bt.bt_fit_chebyshev(Gn, hn, rel_err=1e-6)
    assert loss > 0 and true(c) < 10 * true(c_exact) + 1e-6
    assert abs(loss - true(c)) < 0.1 * true(c) + 1e-6
    _, _, c_bad, loss_bad = bt.bt_fit_chebyshev(Gn, hn, rel_err=1e-14)
    assert loss_bad < 0.5 * true(c_bad) and true(c_bad) > 5 * true(c)


def test_fit_refuses_empty_or_bad_data():
    with pytest.raises(bt.BtError):
        bt.bt_fit_chebyshev(np.full((1, 81), np.nan), np.zeros((1, 9)))
    with pytest.raises(bt.BtError):
        bt.bt_fit_chebyshev(np.eye(9)[None], np.ones((1, 9)), rel_err=-1.0)

"""Matrix-formalism signal of the 1-D Neumann interval (test infrastructure only).

The paper validates its finite-element signals against matrix-formalism
reference signals (Section 4, Figs. 5-7).  For free diffusion in a box with
homogeneous Neumann walls and the gradient along x, the Bloch-Torrey solution
(Eq. strong_BT) with uniform initial magnetisation depends on x only, so the
signal equals that of the interval [-L/2, L/2].  In the Neumann eigenbasis
phi_0 = 1/sqrt(L), phi_m = sqrt(2/L) cos(m pi (x + L/2) / L), eigenvalues
lambda_m = D (m pi / L)^2, the coefficients obey
    dc/dt = -(Lambda + i q f(t) X) c,   X_mn = integral x phi_m phi_n dx,
and for the piecewise-constant PGSE profile (Eq. pgse) the signal ratio is
    S/S0 = e_0^T  exp(-(Lambda - i q X) delta) exp(-Lambda (Delta - delta))
                  exp(-(Lambda + i q X) delta)  e_0.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def moment_matrix(L: float, n_modes: int):
    """X_mn = integral_{-L/2}^{L/2} x phi_m(x) phi_n(x) dx in closed form:
    zero unless m + n is odd, then -c_m c_n (L/pi)^2 (1/(m-n)^2 + 1/(m+n)^2)
    with c_0 = 1/sqrt(L), c_m = sqrt(2/L)."""
    m = np.arange(n_modes)
    c = np.where(m == 0, 1.0 / np.sqrt(L), np.sqrt(2.0 / L))
    mm, nn = np.meshgrid(m, m, indexing="ij")
    odd = (mm + nn) % 2 == 1
    with np.errstate(divide="ignore", invalid="ignore"):
        val = -(L / np.pi) ** 2 * (1.0 / (mm - nn) ** 2 + 1.0 / (mm + nn) ** 2)
    return np.where(odd, c[:, None] * c[None, :] * val, 0.0)


def mf_interval_signal(L: float, D: float, q: float, delta: float, Delta: float,
                       n_modes: int = 400) -> complex:
    m = np.arange(n_modes)
    lam = np.diag(D * (m * np.pi / L) ** 2)
    X = moment_matrix(L, n_modes)
    E1 = sla.expm(-(lam + 1j * q * X) * delta)
    E2 = sla.expm(-lam * (Delta - delta))
    E3 = sla.expm(-(lam - 1j * q * X) * delta)
    c = np.zeros(n_modes, dtype=complex)
    c[0] = 1.0
    return complex((E3 @ (E2 @ (E1 @ c)))[0])

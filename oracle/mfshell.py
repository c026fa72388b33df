"""Matrix-formalism signal of diffusion on a spherical shell (test
infrastructure only): the thin-layer limit of the paper's multilayer spheres.

On the sphere of radius R the Laplace-Beltrami eigenfunctions are the
spherical harmonics Y_lm with eigenvalues lambda_l = D l (l + 1) / R^2.  From
the uniform magnetisation with the gradient along z only the zonal family
Y_l0 is reached, and z = R cos(theta) couples l to l + 1 with
    <Y_l0 | cos theta | Y_{l+1,0}> = (l + 1) / sqrt((2 l + 1)(2 l + 3))
(the recurrence of the Legendre polynomials).  For the PGSE profile
(Eq. pgse) the signal ratio is then
    S/S0 = e_0^T exp(-(Lambda - i q X) delta) exp(-Lambda (Delta - delta))
                 exp(-(Lambda + i q X) delta) e_0.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def moment_matrix(R: float, L: int):
    """X_ab = integral z Y_a0 Y_b0 dA / integral Y_a0^2 dA for l = 0..L-1."""
    X = np.zeros((L, L))
    for l in range(L - 1):
        X[l, l + 1] = X[l + 1, l] = R * (l + 1) / np.sqrt((2 * l + 1) * (2 * l + 3))
    return X


def mf_shell_signal(R: float, D: float, q: float, delta: float, Delta: float, L: int = 60) -> complex:
    l = np.arange(L)
    lam = np.diag(D * l * (l + 1) / R ** 2)
    X = moment_matrix(R, L)
    E1 = sla.expm(-(lam + 1j * q * X) * delta)
    E2 = sla.expm(-lam * (Delta - delta))
    E3 = sla.expm(-(lam - 1j * q * X) * delta)
    c = np.zeros(L, dtype=complex)
    c[0] = 1.0
    return complex((E3 @ (E2 @ (E1 @ c)))[0])

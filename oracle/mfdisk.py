"""Matrix-formalism signal of the Neumann disk (test infrastructure only).

The paper checks its two-dimensional disk signals against matrix-formalism
reference values (Section 4).  For free diffusion in a disk of radius R with
homogeneous Neumann walls, the Laplacian eigenfunctions are
    phi_nk = J_n(alpha_nk r / R) cos(n theta) / N_nk   (and the sine family),
with alpha_nk the zeros of J_n' (alpha_00 = 0, the constant mode) and
eigenvalues lambda_nk = D alpha_nk^2 / R^2.  Starting from the uniform
magnetisation with the gradient along x, only the cosine family is reached.
In that basis the Bloch-Torrey equation (Eq. strong_BT) reads
    dc/dt = -(Lambda + i q f(t) X) c,   X_ab = integral x phi_a phi_b dA,
and for the PGSE profile (Eq. pgse) the signal ratio is
    S/S0 = e_0^T exp(-(Lambda - i q X) delta) exp(-Lambda (Delta - delta))
                 exp(-(Lambda + i q X) delta) e_0.
The radial integrals are done by Gauss-Legendre quadrature and the angular
ones by the trapezoid rule (exact for the trigonometric polynomials involved):
a route independent of the finite-element code.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.special as sps


def _modes(n_ang: int, n_rad: int):
    """(n, alpha) of the cosine family, n = 0..n_ang, n_rad radial modes each."""
    out = []
    for n in range(n_ang + 1):
        if n == 0:
            al = np.concatenate([[0.0], sps.jnp_zeros(0, n_rad - 1)])
        else:
            al = sps.jnp_zeros(n, n_rad)
        out += [(n, float(a)) for a in al]
    return out


def moment_matrix(R: float, n_ang: int, n_rad: int, n_quad: int = 600):
    """(alpha, X): the eigenvalue roots and X_ab = integral x phi_a phi_b dA."""
    modes = _modes(n_ang, n_rad)
    xg, wg = np.polynomial.legendre.leggauss(n_quad)
    r = 0.5 * R * (xg + 1.0)
    w = 0.5 * R * wg
    J = np.array([sps.jv(n, a * r / R) for n, a in modes])              # [m, nq]
    ns = np.array([n for n, _ in modes])
    # angular integrals by the trapezoid rule on enough points to be exact
    M = 4 * n_ang + 8
    th = 2.0 * np.pi * np.arange(M) / M
    C = np.cos(np.outer(np.arange(n_ang + 1), th))                      # [n_ang+1, M]
    ang_norm = (2.0 * np.pi / M) * np.sum(C * C, axis=1)                # 2 pi (n = 0), pi (n > 0)
    ang_x = (2.0 * np.pi / M) * np.einsum("am,bm,m->ab", C, C, np.cos(th))
    rad_norm = np.sum(w * r * J * J, axis=1)
    N = np.sqrt(ang_norm[ns] * rad_norm)
    rad_x = np.einsum("q,aq,bq->ab", w * r * r, J, J)
    X = ang_x[np.ix_(ns, ns)] * rad_x / np.outer(N, N)
    return np.array([a for _, a in modes]), X


def mf_disk_signal(R: float, D: float, q: float, delta: float, Delta: float,
                   n_ang: int = 24, n_rad: int = 24) -> complex:
    alpha, X = moment_matrix(R, n_ang, n_rad)
    lam = np.diag(D * alpha ** 2 / R ** 2)
    E1 = sla.expm(-(lam + 1j * q * X) * delta)
    E2 = sla.expm(-lam * (Delta - delta))
    E3 = sla.expm(-(lam - 1j * q * X) * delta)
    c = np.zeros(len(alpha), dtype=complex)
    c[0] = 1.0
    return complex((E3 @ (E2 @ (E1 @ c)))[0])

"""FP64 CPU reference of the learned polynomial preconditioner (test
infrastructure only).

Model (a learned preconditioner added to the method: the paper itself leaves
the linear solver to an unnamed PETSc method, Appendix B "linsolver"):
  features  phi = (dt, q |f|, D, kappa, h), each mapped to
            x_k = (log(phi_k + eps_k) - mu_k) / sd_k  (constants FEATURE_NORM)
  network   a1 = relu(W1 x + b1) (64), a2 = relu(W2 a1 + b2) (64),
            c = W3 a2 + b3 (9); weights rounded to bfloat16 when bf16=True
  precond   P_c = sum_{j=0}^{8} c_j B^j D^-1,  B = D^-1 A, D = diag(A)
  data      for a right-hand side r: v_0 = D^-1 r, v_j = B v_{j-1},
            y_j = A v_j;  G = Re(Y^H Y)/|r|^2 (9x9), h = Re(Y^H r)/|r|^2 (9)
  loss      L(c) = |r - A P_c r|^2 / |r|^2 = 1 - 2 c^T h + c^T G c,
            averaged over samples; its per-sample minimum is c* = G^-1 h.
The parameters are one flat vector in the order W1 (64x5, row-major), b1, W2
(64x64), b2, W3 (9x64), b3 -- the same order the CUDA library uses.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 5, 64, 9
N_PARAM = N_H * N_IN + N_H + N_H * N_H + N_H + N_OUT * N_H + N_OUT
# eps, mu, sd per feature: dt [us], q|f| [rad/(um us)] or q|F| [rad/um], D [um^2/us], kappa [um/us], h [um]
FEATURE_NORM = np.array([
    [1e-3, 3.9, 0.5],
    [1e-6, -10.0, 2.0],
    [1e-6, -6.2, 0.3],
    [1e-8, -10.4, 0.7],
    [1e-3, -0.5, 0.7],
])


def normalise(phi):
    phi = np.atleast_2d(np.asarray(phi, float))
    return (np.log(phi + FEATURE_NORM[:, 0]) - FEATURE_NORM[:, 1]) / FEATURE_NORM[:, 2]


def unpack(w):
    w = np.asarray(w, float)
    o = 0
    out = []
    for shape in [(N_H, N_IN), (N_H,), (N_H, N_H), (N_H,), (N_OUT, N_H), (N_OUT,)]:
        k = int(np.prod(shape))
        out.append(w[o:o + k].reshape(shape))
        o += k
    return out


def bf16_round(a):
    """Round FP64 values to the nearest bfloat16 (ties to even), via FP32."""
    f = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> 16) & 1
    r = ((f + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(w, x, bf16=True):
    W1, b1, W2, b2, W3, b3 = unpack(bf16_round(w) if bf16 else w)
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    c = a2 @ W3.T + b3
    return c, (x, z1, a1, z2, a2)


def loss_and_grad(w, x, G, h, bf16=True, rel_err=0.0):
    """Mean loss over samples and its gradient with respect to the flat
    parameters (through the bf16-rounded weights, straight-through).  With
    rel_err > 0 each sample's loss carries its spread for data known to that
    relative accuracy, rel_err (2 |c|.|h| + |c|.|G| |c|): G and h come from
    nearly dependent FP32 Krylov vectors, and a coefficient vector whose loss
    is below that spread is not resolved by the data."""
    W1, b1, W2, b2, W3, b3 = unpack(bf16_round(w) if bf16 else w)
    c, (x, z1, a1, z2, a2) = forward(w, x, bf16)
    n = len(x)
    Gc = np.einsum("sij,sj->si", G, c)
    L = 1.0 - 2.0 * np.sum(c * h, axis=1) + np.sum(c * Gc, axis=1)
    dc = 2.0 * (Gc - h) / n
    if rel_err > 0:
        ac, aGc = np.abs(c), np.einsum("sij,sj->si", np.abs(G), np.abs(c))
        L = L + rel_err * (2.0 * np.sum(ac * np.abs(h), axis=1) + np.sum(ac * aGc, axis=1))
        dc = dc + 2.0 * rel_err * np.sign(c) * (np.abs(h) + aGc) / n
    gW3 = dc.T @ a2
    gb3 = dc.sum(0)
    d2 = (dc @ W3) * (z2 > 0)
    gW2 = d2.T @ a1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ x
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return float(L.mean()), g, L


def optimal_coefficients(G, h):
    """Per-sample minimiser c* = G^-1 h (least squares if G is singular)."""
    return np.stack([np.linalg.lstsq(Gs, hs, rcond=None)[0] for Gs, hs in zip(G, h)])


def gram_data(A, r, degree=8):
    """G, h of one right-hand side r for the (sparse or dense) matrix A."""
    d = A.diagonal()
    v = r / d
    Y = []
    for _ in range(degree + 1):
        y = A @ v
        Y.append(y)
        v = y / d
    Y = np.stack(Y, axis=1)
    nr2 = np.vdot(r, r).real
    G = (Y.conj().T @ Y).real / nr2
    h = (Y.conj().T @ r).real / nr2
    return G, h

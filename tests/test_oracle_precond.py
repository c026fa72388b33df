"""Pins of the CPU reference of the learned polynomial preconditioner
(brute force on small matrices, finite differences, an independent bf16
rounding, optimality of the per-sample minimiser).  CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import precond as pc


def _system(n=40, seed=0):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(n, n)) * 0.1
    A = np.eye(n) * 4 + B + B.T + 1j * 0.3 * np.diag(rng.normal(size=n))  # complex symmetric
    r = rng.normal(size=n) + 1j * rng.normal(size=n)
    return sp.csr_matrix(A), r


def test_loss_identity_brute_force():
    A, r = _system()
    G, h = pc.gram_data(A, r)
    rng = np.random.default_rng(1)
    c = rng.normal(size=9)
    # P_c r = sum_j c_j B^j D^-1 r, evaluated directly
    d = A.diagonal()
    Ad = A.toarray()
    B = Ad / d[:, None]
    v = r / d
    Pr = np.zeros_like(r)
    for j in range(9):
        Pr = Pr + c[j] * v
        v = B @ v
    direct = np.linalg.norm(r - Ad @ Pr) ** 2 / np.linalg.norm(r) ** 2
    assert abs(direct - (1 - 2 * c @ h + c @ G @ c)) < 1e-10 * max(1.0, direct)
    # c = e_0 is one Jacobi step
    jac = np.linalg.norm(r - Ad @ (r / d)) ** 2 / np.linalg.norm(r) ** 2
    e0 = np.eye(9)[0]
    assert abs(jac - (1 - 2 * e0 @ h + e0 @ G @ e0)) < 1e-12


@pytest.mark.parametrize("rel_err", [0.0, 1e-3])
def test_gradient_matches_finite_differences(rel_err):
    """The objective's gradient (the plain loss, and the loss with its spread
    for data of relative accuracy rel_err) against central differences."""
    rng = np.random.default_rng(2)
    w = rng.normal(size=pc.N_PARAM) * 0.2
    ns = 7
    x = rng.normal(size=(ns, 5))
    G, h = [], []
    for s in range(ns):
        A, r = _system(20, seed=10 + s)
        g_, h_ = pc.gram_data(A, r)
        G.append(g_)
        h.append(h_)
    G, h = np.array(G), np.array(h)
    L, g, _ = pc.loss_and_grad(w, x, G, h, bf16=False, rel_err=rel_err)
    idx = rng.choice(pc.N_PARAM, 60, replace=False)
    eps = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        fd = (pc.loss_and_grad(wp, x, G, h, bf16=False, rel_err=rel_err)[0] -
              pc.loss_and_grad(wm, x, G, h, bf16=False, rel_err=rel_err)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    if rel_err:
        # the added term, summed element by element
        c = pc.forward(w, x, bf16=False)[0]
        extra = 0.0
        for s_ in range(ns):
            for i in range(9):
                extra += 2 * abs(c[s_, i]) * abs(h[s_, i])
                for j in range(9):
                    extra += abs(c[s_, i]) * abs(G[s_, i, j]) * abs(c[s_, j])
        L0 = pc.loss_and_grad(w, x, G, h, bf16=False)[0]
        assert abs(L - L0 - rel_err * extra / ns) <= 1e-12 * max(1.0, abs(L))


def test_optimal_coefficients_minimise_loss():
    A, r = _system(30, seed=4)
    G, h = pc.gram_data(A, r)
    c = pc.optimal_coefficients(G[None], h[None])[0]
    L0 = 1 - 2 * c @ h + c @ G @ c
    rng = np.random.default_rng(5)
    for _ in range(20):
        d = rng.normal(size=9) * 1e-3
        c2 = c + d
        assert 1 - 2 * c2 @ h + c2 @ G @ c2 >= L0 - 1e-12
    assert L0 < 1.0


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    a = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 0.0]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(pc.bf16_round(a), ref)

"""GPU tests of the learned polynomial preconditioner: the library's own
forward/backward kernels against the FP64 CPU reference (oracle/precond.py),
its training-data collection against the oracle's Gram data, training, and
the LEARNED run mode, whose signals are compared one by one with the FP64
oracle (1e-6 relative), live and on a stored oracle case."""
import numpy as np
import pytest
import scipy.sparse as sp

import geom
import oracle
from oracle import btoracle as bo
from oracle import precond as pc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    from paper_1908_01719_gb300 import build, bt as btmod
    build.build()
    return btmod


@pytest.fixture(scope="module")
def sim_cls(bt):
    from paper_1908_01719_gb300.simulate import Simulation
    return Simulation


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    feat = np.stack([rng.uniform(20, 100, n), rng.uniform(0, 3e-4, n), rng.uniform(1e-3, 3e-3, n),
                     rng.uniform(1e-5, 1e-4, n), rng.uniform(0.3, 2.0, n)], axis=1).astype(np.float32)
    G, h = [], []
    for s in range(n):
        m = 12
        B = rng.normal(size=(m, m)) * 0.1
        A = np.eye(m) * 3 + B + B.T + 1j * 0.2 * np.diag(rng.normal(size=m))
        r = rng.normal(size=m) + 1j * rng.normal(size=m)
        g_, h_ = pc.gram_data(sp.csr_matrix(A), r)
        G.append(g_)
        h.append(h_)
    return feat, np.array(G), np.array(h)


def test_forward_and_gradient_match_cpu_reference(sim_cls, bt):
    p = geom.cfg1(n=2)
    sim = sim_cls(p)
    try:
        rng = np.random.default_rng(3)
        w = (rng.normal(size=bt.BT_PRECOND_NPARAM) * 0.2).astype(np.float32)
        bt.bt_load_precond(sim.ctx, w)
        assert np.array_equal(bt.bt_save_precond(sim.ctx), w)
        feat, G, h = _samples(64, 4)
        x = pc.normalise(feat.astype(np.float64))
        c_ref, _ = pc.forward(w.astype(np.float64), x, bf16=True)
        for rel_err in (0.0, 1e-3):  # the plain loss, and the loss with its data spread
            coef, loss, grad = bt.bt_precond_eval(sim.ctx, feat, G, h, rel_err=rel_err)
            L_ref, g_ref, _ = pc.loss_and_grad(w.astype(np.float64), x, G, h, bf16=True, rel_err=rel_err)
            assert np.abs(coef - c_ref).max() <= 1e-4 * np.abs(c_ref).max()
            assert abs(loss - L_ref) <= 1e-4 * abs(L_ref)
            assert np.linalg.norm(grad - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
    finally:
        sim.close()


def test_collected_gram_data_matches_oracle(sim_cls, bt):
    """Step 1 of a lab-frame run: r_0 = (R_1 - L_1) 1; the library's Krylov
    basis of the normalised r_0 gives the oracle's G and h."""
    p = geom.cfg2(n=6, kappa=1e-4, bvals=(1000.0, 3000.0))
    sim = sim_cls(p)
    try:
        feat, G, h = bt.bt_collect_precond_data(sim.ctx, [1], p.n_rhs)
        a = bo.assemble(p)
        fbar, _ = oracle.pgse_tables(p.delta, p.Delta, p.dt, p.n_steps)
        for r in range(p.n_rhs):
            q = float(oracle.q_from_b(p.bvals[r % len(p.bvals)], p.delta, p.Delta))
            qh = p.dirs[r // len(p.bvals)]
            Mq = qh[0] * a["Mx"] + qh[1] * a["My"] + qh[2] * a["Mz"]
            A = a["K"] + a["J"] + 1j * q * fbar[0] * Mq
            L = (a["M"] + 0.5 * p.dt * A).tocsr()
            r0 = -p.dt * (A @ np.ones(a["n"]))
            Gr, hr = pc.gram_data(L, r0)
            assert np.abs(G[r] - Gr).max() <= 2e-4 * np.abs(Gr).max()
            assert np.abs(h[r] - hr).max() <= 2e-4 * np.abs(hr).max()
            assert abs(feat[r, 1] - q) <= 1e-6 * q and abs(feat[r, 0] - p.dt) < 1e-3
    finally:
        sim.close()


@pytest.fixture(scope="module")
def trained(sim_cls, bt):
    """A network trained on step solves of a small seeded packing."""
    p = geom.cfg4(n=16, n_dir=8, bvals=(500.0, 1000.0, 2000.0, 3000.0))
    sim = sim_cls(p)
    steps = [1, 10, 25, 50, 51, 75, 100, 101, 120, 150]
    feat, G, h = bt.bt_collect_precond_data(sim.ctx, steps, p.n_rhs)
    ok = np.abs(G).sum(axis=(1, 2)) > 0
    feat, G, h = feat[ok], G[ok], h[ok]
    hist = bt.bt_train_precond(sim.ctx, feat, G, h, bt.bt_train_default_opts(epochs=200, batch=64))
    return p, sim, feat, G, h, hist


def test_training_reduces_loss_above_optimum(trained, bt):
    p, sim, feat, G, h, hist = trained
    assert hist[-1] < 0.5 * hist[0] or hist[-1] < hist[0] - 0.01
    coef, loss, _ = bt.bt_precond_eval(sim.ctx, feat, G, h)
    cstar = pc.optimal_coefficients(G, h)
    Lstar = np.mean(1 - 2 * np.sum(cstar * h, 1) + np.einsum("si,sij,sj->s", cstar, G, cstar))
    e0 = np.eye(9)[0]
    Ljac = np.mean(1 - 2 * h @ e0 + np.einsum("i,sij,j->s", e0, G, e0))
    assert Lstar - 1e-6 <= loss < Ljac


def test_learned_mode_matches_oracle(trained, bt):
    """The learned-preconditioned mixed solve is judged by the same refinement
    tolerance as Jacobi, so each of its signals must match the FP64 oracle to
    1e-6 relative (per signal, not scaled by the largest one)."""
    p, sim, *_ = trained
    S_j, err_j, st_j, _ = sim.run(bt.BT_MODE_MIXED)
    it_j = sim.stats()["krylov_iters"]
    S_l, err_l, st_l, _ = sim.run(bt.BT_MODE_LEARNED)
    it_l = sim.stats()["krylov_iters"]
    assert np.all(st_j == 0) and np.all(st_l == 0)
    # a sample over directions and all four b-values (b = 500 ... 3000)
    rhs = [0, 5, 10, 15, 18, 23, 28, 31]
    ref = np.asarray(oracle.run(p, rhs=rhs))
    e_l = np.abs(S_l[rhs] - ref) / np.abs(ref)
    e_j = np.abs(S_j[rhs] - ref) / np.abs(ref)
    print(f"Krylov iterations: Jacobi {it_j}, learned polynomial {it_l}; "
          f"max rel err vs oracle: learned {e_l.max():.2e}, Jacobi {e_j.max():.2e}")
    assert e_l.max() < 1e-6, e_l
    assert e_j.max() < 1e-6, e_j
    assert it_l < it_j   # the trained polynomial needs fewer (but costlier) iterations


def test_fixed_chebyshev_matches_oracle(trained, bt):
    """The fixed Chebyshev polynomial, its interval fitted to the same samples,
    runs through the same Horner kernels: fewer Krylov iterations than Jacobi,
    8 + 1 Horner launches per polynomial application, signals within 1e-6 of
    the FP64 oracle; with the fixed polynomial cleared the network runs again."""
    p, sim, feat, G, h, _ = trained
    lo, hi, c, loss = bt.bt_fit_chebyshev(G, h)
    e0 = np.eye(9)[0]
    Ljac = np.mean(1 - 2 * h @ e0 + np.einsum("i,sij,j->s", e0, G, e0))
    assert 0 < lo < hi and loss < Ljac
    sim.run(bt.BT_MODE_MIXED)
    it_j = sim.stats()["krylov_iters"]
    bt.bt_set_precond_poly(sim.ctx, c)
    try:
        S_c, _, st_c, _ = sim.run(bt.BT_MODE_LEARNED)
        it_c = sim.stats()["krylov_iters"]
        hor = bt.bt_get_precond_stats(sim.ctx)["horner_launches"]
    finally:
        bt.bt_set_precond_poly(sim.ctx, None)
    assert np.all(st_c == 0) and it_c < it_j
    assert hor > 0 and hor % 9 == 0
    rhs = [0, 7, 13, 22, 31]
    ref = np.asarray(oracle.run(p, rhs=rhs))
    e = np.abs(S_c[rhs] - ref) / np.abs(ref)
    print(f"Chebyshev on [{lo:.3g}, {hi:.3g}], mean loss {loss:.3g} (Jacobi {Ljac:.3g}); "
          f"Krylov iterations {it_c} vs Jacobi {it_j}; max rel err vs oracle {e.max():.2e}")
    assert e.max() < 1e-6, e
    sim.run(bt.BT_MODE_LEARNED)
    assert bt.bt_get_precond_stats(sim.ctx)["horner_launches"] > 0


def test_fixed_polynomial_needs_no_network(sim_cls, bt):
    """A context without a network runs BT_MODE_LEARNED on a fixed polynomial
    and matches the oracle; NULL coefficients bring back the refusal."""
    p = geom.cfg1(n=4)
    sim = sim_cls(p)
    try:
        bt.bt_set_precond_poly(sim.ctx, bt.bt_chebyshev_poly(0.05, 2.5))
        S, _, st, _ = sim.run(bt.BT_MODE_LEARNED)
        assert np.all(st == 0)
        ref = np.asarray(oracle.run(p))
        assert np.max(np.abs(S - ref) / np.abs(ref)) < 1e-6
        with pytest.raises(bt.BtError):
            bt.bt_set_precond_poly(sim.ctx, np.full(9, np.nan))
        bt.bt_set_precond_poly(sim.ctx, None)
        with pytest.raises(bt.BtError) as e:
            sim.run(bt.BT_MODE_LEARNED)
        assert e.value.code == bt.BT_ESTATE
    finally:
        sim.close()


def test_learned_mode_golden_signals(trained, sim_cls, bt):
    """The trained network, loaded into a context of the 24^3 packing, runs the
    stored oracle case of that geometry in LEARNED mode (per signal 1e-6)."""
    import json
    import os
    _, sim_t, *_ = trained
    w = bt.bt_save_precond(sim_t.ctx)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg4_n24.json")
    with open(path) as f:
        g = json.load(f)
    p = getattr(geom, g["builder"])(**g["kwargs"])
    ref = np.array(g["S_re"]) + 1j * np.array(g["S_im"])
    sim = sim_cls(p)
    try:
        bt.bt_load_precond(sim.ctx, w)
        S = np.zeros(len(g["rhs"]), complex)
        for k, r in enumerate(g["rhs"]):
            Sk, err, stat, _ = sim.run(bt.BT_MODE_LEARNED, rhs_begin=r, rhs_end=r + 1)
            assert stat[r] == 0
            S[k] = Sk[r]
        e = np.abs(S - ref) / np.abs(ref)
        assert e.max() < 1e-6, e
    finally:
        sim.close()


def test_learned_mode_requires_network(sim_cls, bt):
    p = geom.cfg1(n=3)
    sim = sim_cls(p)
    try:
        with pytest.raises(bt.BtError) as e:
            sim.run(bt.BT_MODE_LEARNED)
        assert e.value.code == bt.BT_ESTATE
    finally:
        sim.close()

"""Pins of the 1-D manifold (P1 segment) discretisation.  The element
matrices are checked against Gauss quadrature along the segment; a straight
fibre against the matrix formalism of the Neumann interval (second order in h
and dt together); the embedding against rotation (only the projection of the
gradient on the fibre matters, an exact discrete identity); a branched tree
against its length, linear fields and conservation at g = 0."""

import numpy as np
import pytest

import geom
import oracle
from oracle import btoracle as bo


def _one_segment(X0, X1, D=2e-3, centre=(0.3, -0.2, 0.5)):
    p = geom.line_segments(1)
    p.xyz = np.array([X0, X1], float)
    c = np.asarray(centre, float)
    p.box_lo, p.box_hi = c - 10.0, c + 10.0
    p.D_cmpt = np.array([D])
    return p


def test_segment_matrices_by_quadrature():
    rng = np.random.default_rng(3)
    X0, X1 = rng.normal(size=3), rng.normal(size=3) * 2.0
    D = 1.7e-3
    p = _one_segment(X0, X1, D)
    a = bo.assemble(p)
    e = X1 - X0
    ell = np.linalg.norm(e)
    t = e / ell
    c = 0.5 * (p.box_lo + p.box_hi)
    s, w = np.polynomial.legendre.leggauss(6)
    s, w = 0.5 * (s + 1), 0.5 * w
    phi = np.stack([1 - s, s])                       # [2, nq]
    dphi = np.array([-1.0, 1.0]) / ell               # derivative along arclength
    x = X0[None] + s[:, None] * e[None]              # [nq, 3]
    M = np.einsum("q,iq,jq->ij", w, phi, phi) * ell
    K = D * np.outer(dphi, dphi) * ell
    ref = {"M": M, "K": K, "MD": D * M}
    for k, nm in enumerate("xyz"):
        ref["M" + nm] = np.einsum("q,iq,jq,q->ij", w, phi, phi, x[:, k] - c[k]) * ell
        C = D * np.einsum("q,iq,j->ij", w, phi, dphi * t[k]) * ell     # D int phi_i d_k phi_j
        ref["E" + nm] = C - C.T
    for nm, R in ref.items():
        A = a[nm].toarray()
        assert np.abs(A - R).max() < 1e-15 * max(1.0, np.abs(R).max()) + 1e-17, nm
    assert a["n_iface"] == 0 and a["J"].count_nonzero() == 0


def test_straight_fibre_converges_to_interval_matrix_formalism():
    """A fibre along x is the Neumann interval: second-order convergence to
    the matrix-formalism signal (the published worked value 0.1997576)."""
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    ref = oracle.mf_interval_signal(40.0, 2e-3, q, 2500.0, 5000.0, 400).real
    errs = []
    for n, dt in [(48, 50.0), (96, 25.0), (192, 12.5)]:
        S = oracle.run(geom.line_segments(n, dt=dt))[0] / 40.0
        errs.append(abs(S.real - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_only_the_projection_on_the_fibre_matters():
    """Fibre along t with gradient direction qhat at b equals the fibre along x
    with the gradient along x at b (qhat.t)^2: M_k = t_k M_s for a straight
    fibre through the centre, so the step matrices coincide."""
    t = np.array([0.36, 0.48, 0.8])
    qh = np.array([0.0, 0.6, -0.8])
    b = 2000.0
    S_t = oracle.run(geom.line_segments(40, direction=t, dirs=(qh,), bvals=(b,)))[0]
    S_x = oracle.run(geom.line_segments(40, bvals=(b * float(qh @ t) ** 2,)))[0]
    assert abs(S_t - S_x) < 1e-12 * abs(S_x)
    # and a direction orthogonal to the fibre sees no gradient at all
    S_0 = oracle.run(geom.line_segments(40, direction=t, dirs=((0.8, -0.6, 0.0),), bvals=(b,)))[0]
    assert abs(S_0 - 40.0) < 1e-12 * 40.0


@pytest.fixture(scope="module")
def tree():
    p = geom.dendrite_tree(seed=1, n_stems=3, depth=3, length=(8.0, 15.0))
    return p, bo.assemble(p)


def test_tree_length_linear_fields_and_symmetry(tree):
    p, a = tree
    n = a["n"]
    one = np.ones(n)
    seg_len = np.linalg.norm(p.xyz[p.tets[:, 1]] - p.xyz[p.tets[:, 0]], axis=1)
    assert n == len(p.xyz)                                 # no doubling on a manifold
    assert abs(one @ a["M"] @ one - seg_len.sum()) < 1e-12 * seg_len.sum()
    assert np.abs(a["K"] @ one).max() < 1e-14
    X = p.xyz[a["dof_node"]]
    c = 0.5 * (p.box_lo + p.box_hi)
    rng = np.random.default_rng(0)
    for _ in range(3):
        g = rng.normal(size=3)
        u = X @ g
        # energy of a linear field: D sum over segments of (g.e)^2 / |e|
        e = p.xyz[p.tets[:, 1]] - p.xyz[p.tets[:, 0]]
        assert abs(u @ a["K"] @ u - 2e-3 * np.sum((e @ g) ** 2 / seg_len)) < 1e-10 * abs(u @ a["K"] @ u)
    for k, nm in enumerate("xyz"):
        # int (x_k - c_k) along the tree = sum |e| (midpoint_k - c_k), and int x_k^2 by Simpson per segment
        mid = 0.5 * (p.xyz[p.tets[:, 0], k] + p.xyz[p.tets[:, 1], k]) - c[k]
        assert abs(one @ a["M" + nm] @ one - np.sum(seg_len * mid)) < 1e-9 * np.sum(seg_len * np.abs(mid))
        E = a["E" + nm]
        assert abs(E + E.T).max() < 1e-18
        assert abs(a["M" + nm] - a["M" + nm].T).max() < 1e-14


def test_tree_conserves_at_zero_gradient(tree):
    p, a = tree
    p.bvals = np.array([0.0])
    seg_len = np.linalg.norm(p.xyz[p.tets[:, 1]] - p.xyz[p.tets[:, 0]], axis=1)
    S, H = oracle.run(p, return_history=True)
    assert np.abs(H[0] - seg_len.sum()).max() < 1e-10 * seg_len.sum()


def test_manifold_refusals():
    p = geom.line_segments(8)
    p.transformed = True
    with pytest.raises(ValueError):
        bo.assemble(p)
    q = geom.line_segments(8)
    q.tet_cmpt = np.array([0, 0, 0, 0, 1, 1, 1, 1], np.int32)   # compartments meet at node 4
    q.D_cmpt, q.kappa_cmpt = np.array([2e-3, 1e-3]), np.array([1e-4, 1e-4])
    with pytest.raises(ValueError):
        bo.assemble(q)

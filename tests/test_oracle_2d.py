"""Pins of the 2-D (P1 triangle) discretisation.  The barycentric moments are
checked against direct quadrature on the reference triangle; the assembled
matrices against identities that fix them (areas, linear fields, moments,
skew-symmetry, the interface length measured independently); the whole
2-D transformed path against the exact discrete solution of free diffusion
in a periodic square; the lab path by conservation at g = 0."""
import math

import numpy as np
import pytest

import geom
import oracle
from oracle import btoracle as bo


def test_triangle_cubic_moments_by_quadrature():
    """int over the reference triangle of l_i l_j l_l / area, by a Duffy map of
    Gauss-Legendre points (exact for these cubics)."""
    x, w = np.polynomial.legendre.leggauss(8)
    u, v = np.meshgrid(0.5 * (x + 1), 0.5 * (x + 1), indexing="ij")
    W = np.outer(0.25 * w, w)
    s, t = u * (1 - v), u * v                  # Duffy: Jacobian u
    lam = [1 - s - t, s, t]
    c = bo._cubic_moments(2)
    for i in range(3):
        for j in range(3):
            for l in range(3):
                q = np.sum(W * u * lam[i] * lam[j] * lam[l]) / 0.5
                assert abs(q - c[i, j, l]) < 1e-14


@pytest.fixture(scope="module")
def disk():
    p = geom.square_disk(n=12, L=10.0, R=3.0)
    return p, bo.assemble(p)


def test_area_linear_fields_and_moments(disk):
    p, a = disk
    n = a["n"]
    one = np.ones(n)
    assert abs(one @ a["M"] @ one - 100.0) < 1e-12 * 100.0
    for nm in ("K", "J"):
        assert np.abs(a[nm] @ one).max() < 1e-14
    X = p.xyz[a["dof_node"]]
    # int x_k over the square is 0 (centred); int x^2 = L^4 / 12 by the linear-field identity
    for k, nm in enumerate("xy"):
        assert abs(one @ a["M" + nm] @ one) < 1e-12
        assert abs(X[:, k] @ a["M"] @ X[:, k] - 10.0 ** 4 / 12.0) < 1e-9
        # energy of a linear field: D |grad|^2 area
        assert abs(X[:, k] @ a["K"] @ X[:, k] - 2e-3 * 100.0) < 1e-12
        E = a["E" + nm]
        assert abs(E + E.T).max() < 1e-18
    assert a["Mz"].count_nonzero() == 0 or abs(a["Mz"]).max() < 1e-18


def test_interface_length_by_brute_force(disk):
    """The jump matrix J carries kappa |e| / 6 (1 + delta) per interface edge;
    1^T J_side 1 over one side equals kappa times the interface length, which is
    recomputed here from edges shared by triangles of different labels."""
    p, a = disk
    edges = {}
    for t, tri in enumerate(p.tets):
        for e in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
            edges.setdefault(tuple(sorted(e)), []).append(p.tet_cmpt[t])
    length = sum(np.linalg.norm(p.xyz[i] - p.xyz[j]) for (i, j), c in edges.items() if len(c) == 2 and c[0] != c[1])
    side = (a["dof_cmpt"] == 1).astype(float)
    assert abs(-(side @ a["J"] @ (1 - side)) - 1e-5 * length) < 1e-15 * max(1.0, length)


def test_conservation_at_zero_gradient(disk):
    p, _ = disk
    p.bvals = np.array([0.0])
    S, H = oracle.run(p, return_history=True)
    assert np.max(np.abs(H[0] - 100.0)) < 1e-10 * 100.0


def test_periodic_square_exact_discrete_product():
    """Free diffusion in a periodic square, transformed frame: u stays constant
    and S/|Omega| = prod (1 - (1-th) dt D q^2 F_{n-1}^2) / (1 + th dt D q^2 F_n^2),
    tending to exp(-b D)."""
    errs = []
    for dt in (50.0, 25.0):
        p = geom.free_periodic_square(n=4, L=6.0, dt=dt, dirs=((0.6, 0.8, 0.0),), bvals=(900.0,))
        S = oracle.run(p)[0] / 36.0
        fbar, F, I = oracle.sequence(p)
        q2 = 900.0 / I
        prod = np.prod((1 - 0.5 * dt * 2e-3 * q2 * F[:-1] ** 2) / (1 + 0.5 * dt * 2e-3 * q2 * F[1:] ** 2))
        assert abs(S - prod) < 1e-12
        errs.append(abs(S.real - math.exp(-900.0 * 2e-3)))
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_layered_disk_initial_condition_conservation_and_linearity():
    """The paper's three-layer disk (radii 5, 7.5, 10 um) with initial
    magnetization [0, 1, 0]: at g = 0 the signal stays the middle layer's area
    while the membranes exchange magnetization; at any b the scheme is linear
    in the initial condition, S[0,1,0] + S[1,0,1] = S[1,1,1]."""
    p = geom.layered_disk(n=20, bvals=(0.0,))
    X = p.xyz[p.tets]
    area = 0.5 * np.abs(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])[:, 2])
    S, H = oracle.run(p, return_history=True)
    mid = area[p.tet_cmpt == 1].sum()
    assert np.max(np.abs(H[0] - mid)) < 1e-10 * mid
    res = {}
    for rho in ((0.0, 1.0, 0.0), (1.0, 0.0, 1.0), (1.0, 1.0, 1.0)):
        q = geom.layered_disk(n=20, rho=rho, bvals=(1000.0, 4000.0), dirs=((0.6, 0.8, 0.0),))
        res[rho] = oracle.run(q)
    lhs = res[(0.0, 1.0, 0.0)] + res[(1.0, 0.0, 1.0)]
    assert np.max(np.abs(lhs - res[(1.0, 1.0, 1.0)])) < 1e-11 * np.max(np.abs(res[(1.0, 1.0, 1.0)]))
    assert abs(res[(0.0, 1.0, 0.0)][0]) < 0.9 * mid          # the gradient attenuates it


# ---------------------------------------------------------------- the disk against the matrix formalism
def test_disk_matrix_formalism_limits():
    """The disk's matrix formalism: the narrow-pulse long-time limit is the
    closed form [2 J1(k R) / (k R)]^2, k = q delta; no diffusion or no
    gradient leaves the signal at 1; truncation converges."""
    import scipy.special as sps
    from oracle import mfdisk
    R = 5.0
    for k in (0.3, 0.8):
        s = mfdisk.mf_disk_signal(R, 2e-3, k / 1.0, 1.0, 2e6)
        want = (2 * sps.j1(k * R) / (k * R)) ** 2
        assert abs(s - want) < 2e-3 * want, (k, s, want)
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    assert abs(mfdisk.mf_disk_signal(R, 0.0, q, 2500.0, 5000.0) - 1.0) < 1e-10
    assert abs(mfdisk.mf_disk_signal(R, 2e-3, 0.0, 2500.0, 5000.0) - 1.0) < 1e-12
    a = mfdisk.mf_disk_signal(R, 2e-3, q, 2500.0, 5000.0, 16, 16)
    b = mfdisk.mf_disk_signal(R, 2e-3, q, 2500.0, 5000.0, 28, 28)
    assert abs(a - b) < 1e-7


def test_polar_disk_converges_to_matrix_formalism_second_order():
    """P1 triangles on a polar mesh of the disk (boundary nodes on the circle),
    h and dt halved together: the signal approaches the matrix-formalism value
    at second order (error ratios about 4)."""
    from oracle import mfdisk
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    ref = mfdisk.mf_disk_signal(5.0, 2e-3, q, 2500.0, 5000.0).real
    errs = []
    for m, dt in ((8, 50.0), (16, 25.0), (32, 12.5)):
        p = geom.polar_disk(m, dt=dt)
        X = p.xyz[p.tets]
        area = 0.5 * np.abs(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])[:, 2]).sum()
        errs.append(abs(oracle.run(p)[0].real / area - ref))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs

"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
not by the oracle itself: exact integrals, conservation, symmetries, exact
discrete closed forms, brute force on tiny meshes, limits and convergence
orders.  (CPU only.)"""
import copy
import math

import numpy as np
import pytest

import geom
import oracle
from oracle import btoracle as bo
from oracle import mf1d


# ---------------------------------------------------------------- elements
def test_cubic_moments_exact_rationals():
    """integral over the reference tetrahedron of lambda_i lambda_j lambda_l,
    integrated symbolically, equals |T| * c[i,j,l]."""
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    lam = [1 - x - y - z, x, y, z]
    c = bo._cubic_moments()
    for i, j, l in [(0, 0, 0), (1, 1, 2), (0, 2, 3), (3, 3, 1), (2, 2, 2)]:
        e = lam[i] * lam[j] * lam[l]
        val = sympy.integrate(e, (z, 0, 1 - x - y), (y, 0, 1 - x), (x, 0, 1))
        assert abs(float(val) - c[i, j, l] / 6.0) < 1e-15


def test_tet_geometry_reproduces_linear_functions():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(20, 4, 3))
    X[:, 3] += 3.0
    vol, G = bo.tet_geometry(X)
    # volume by the scalar triple product
    e = X[:, 1:] - X[:, :1]
    v2 = np.einsum("ti,ti->t", np.cross(e[:, 0], e[:, 1]), e[:, 2]) / 6.0
    assert np.allclose(vol, v2, rtol=1e-13)
    # gradient of the P1 interpolant of a linear function is exact
    a = rng.normal(size=3)
    f = X @ a + 0.7
    grad = np.einsum("ti,tik->tk", f, G)
    assert np.allclose(grad, a[None, :], atol=1e-12)


def _quad4():
    a, b = 0.5854101966249685, 0.1381966011250105
    return np.array([[a, b, b, b], [b, a, b, b], [b, b, a, b], [b, b, b, a]])


def test_transformed_form_equals_gauge_energy():
    """u^H (K + q^2F^2 MD + i q F Eq) u = sum_T D_T int_T |grad u - i qF qhat u|^2,
    evaluated with a 4-point rule that is exact for quadratics."""
    p = geom.cfg2(n=4)
    p.D_cmpt = np.array([2e-3, 1.3e-3])
    a = bo.assemble(p)
    rng = np.random.default_rng(1)
    u = rng.normal(size=a["n"]) + 1j * rng.normal(size=a["n"])
    qh = np.array([0.3, -0.5, 0.81]); qh /= np.linalg.norm(qh)
    qF = 0.37
    Eq = qh[0] * a["Ex"] + qh[1] * a["Ey"] + qh[2] * a["Ez"]
    A = a["K"] + qF * qF * a["MD"] + 1j * qF * Eq
    lhs = np.vdot(u, A @ u)
    X = p.xyz[p.tets]
    vol, G = bo.tet_geometry(X)
    ue = u[a["tet_dof"]]                       # [nt, 4]
    g = np.einsum("ti,tik->tk", ue, G)         # constant gradient per tet
    B = _quad4()
    uq = ue @ B.T                              # values at the 4 points
    Dt = p.D_cmpt[p.tet_cmpt]
    v = g[:, None, :] - 1j * qF * qh[None, None, :] * uq[:, :, None]
    rhs = np.sum(Dt * vol * 0.25 * np.sum(np.abs(v) ** 2, axis=(1, 2)))
    assert abs(lhs.imag) < 1e-12 * abs(rhs)
    assert abs(lhs.real - rhs) < 1e-12 * abs(rhs)


# ---------------------------------------------------------------- assembly
@pytest.fixture(scope="module")
def sphere_small():
    p = geom.cfg2(n=8, kappa=3e-3)
    return p, bo.assemble(p)


def test_assembly_identities(sphere_small):
    p, a = sphere_small
    one = np.ones(a["n"])
    L = 20.0
    assert abs(one @ a["M"] @ one - L ** 3) < 1e-12 * L ** 3
    assert abs(oracle.signal_weights(a).sum() - L ** 3) < 1e-12 * L ** 3
    for nm in ["K", "J"]:
        assert np.abs(a[nm] @ one).max() < 1e-14 * abs(a[nm]).max() * 20
    for nm in ["M", "K", "J", "Mx", "My", "Mz", "MD"]:
        d = a[nm] - a[nm].T
        assert abs(d).max() <= 1e-15 * max(1.0, abs(a[nm]).max())
    for nm in ["Ex", "Ey", "Ez"]:
        d = a[nm] + a[nm].T
        assert abs(d).max() <= 1e-15 * max(1.0, abs(a[nm]).max())
    # first moments: 1^T M_k 1 = integral of (x_k - centre_k) = 0 for the centred cube
    X = p.xyz[p.tets]
    vol, _ = bo.tet_geometry(X)
    for k, nm in enumerate("xyz"):
        exact = np.sum(vol * (X[:, :, k].mean(axis=1) - 0.0))
        assert abs(one @ a["M" + nm] @ one - exact) < 1e-11
    # D-weighted mass: 1^T MD 1 = sum_c D_c |Omega_c|
    Dv = np.sum(p.D_cmpt[p.tet_cmpt] * vol)
    assert abs(one @ a["MD"] @ one - Dv) < 1e-12 * Dv


def test_first_moment_off_centre():
    """Mesh shifted by s inside a box centred at 0: 1^T M_k 1 = |Omega| s_k."""
    p = geom.cfg1(n=3)
    s = np.array([5.0, -2.0, 1.0])
    p.xyz = p.xyz + s
    a = bo.assemble(p)
    one = np.ones(a["n"])
    for k, nm in enumerate("xyz"):
        assert abs(one @ a["M" + nm] @ one - 64000.0 * s[k]) < 1e-9 * 64000.0


def test_interface_area_brute_force():
    """1_0^T J 1_0 = sum over interface faces of kappa |F|; the faces are found
    here by brute force over all tetrahedron pairs of a tiny mesh."""
    p = geom.cfg2(n=4, kappa=2e-3)
    a = bo.assemble(p)
    side0 = (a["dof_cmpt"] == 0).astype(float)
    lhs = side0 @ a["J"] @ side0
    faces = {}
    for t, tet in enumerate(p.tets):
        for drop in range(4):
            key = tuple(sorted(np.delete(tet, drop)))
            faces.setdefault(key, []).append(t)
    area = 0.0
    for key, ts in faces.items():
        if len(ts) == 2 and p.tet_cmpt[ts[0]] != p.tet_cmpt[ts[1]]:
            X = p.xyz[list(key)]
            area += 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
    kap = 1.0 / (1.0 / math.inf + 1.0 / 2e-3)
    assert area > 0
    assert abs(lhs - kap * area) < 1e-13 * kap * area


def test_periodic_identification_and_skew_annihilates_constants():
    p = geom.free_periodic_box(n=4, L=6.0)
    a = bo.assemble(p)
    assert a["n"] == 4 ** 3
    one = np.ones(a["n"])
    for nm in ["Ex", "Ey", "Ez", "K"]:
        assert np.abs(a[nm] @ one).max() < 1e-15
    assert abs(one @ a["M"] @ one - 216.0) < 1e-12


# ---------------------------------------------------------------- sequence
def test_pgse_tables_and_b_value():
    delta, Delta, dt = 2500.0, 5000.0, 50.0
    N = 150
    fbar, F = oracle.pgse_tables(delta, Delta, dt, N)
    assert set(np.unique(fbar)) == {-1.0, 0.0, 1.0}
    assert np.sum(fbar == 1) == 50 and np.sum(fbar == -1) == 50
    assert abs(F[-1]) < 1e-12 and abs(F[50] - delta) < 1e-12
    # b = q^2 int_0^TE F^2 by fine quadrature of the profile (Eq. b_value)
    t = np.linspace(0, 7500.0, 750001)
    Ft = bo.pgse_F(t, delta, Delta)
    intF2 = np.trapezoid(Ft ** 2, t)
    q = oracle.q_from_b(1000.0, delta, Delta)
    assert abs(q * q * intF2 - 1000.0) < 1e-6 * 1000.0
    assert abs(q - 1.95959e-4) < 1e-9


# ---------------------------------------------------------------- matrix formalism
def test_mf_moment_matrix_closed_form():
    L = 7.0
    X = mf1d.moment_matrix(L, 12)
    xg, wg = np.polynomial.legendre.leggauss(200)
    x = xg * L / 2
    wx = wg * L / 2
    m = np.arange(12)
    phi = np.where(m[:, None] == 0, 1 / np.sqrt(L), np.sqrt(2 / L) * np.cos(m[:, None] * np.pi * (x[None] + L / 2) / L))
    Xq = (phi * x[None] * wx[None]) @ phi.T
    assert np.abs(X - Xq).max() < 1e-12


def test_mf_limits():
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    # no diffusion: the phase refocuses at TE
    assert abs(oracle.mf_interval_signal(40.0, 0.0, q, 2500.0, 5000.0, 200) - 1.0) < 1e-10
    # no gradient
    assert abs(oracle.mf_interval_signal(40.0, 2e-3, 0.0, 2500.0, 5000.0, 50) - 1.0) < 1e-12
    # the published worked value and the approach to exp(-bD) in wide intervals:
    s40 = oracle.mf_interval_signal(40.0, 2e-3, q, 2500.0, 5000.0, 400).real
    assert abs(s40 - 0.1997576) < 2e-7
    gaps = []
    for L in [80.0, 160.0, 320.0]:
        s = oracle.mf_interval_signal(L, 2e-3, q, 2500.0, 5000.0, int(L * 6)).real
        gaps.append(s / math.exp(-2.0) - 1.0)
    assert 0.45 < gaps[1] / gaps[0] < 0.55 and 0.45 < gaps[2] / gaps[1] < 0.55


# ---------------------------------------------------------------- stepping pins
def test_conservation_without_gradient():
    """g = 0, Neumann, permeable interface: 1^T M u^n = |Omega| for all n (P-2)."""
    p = geom.cfg2(n=6, kappa=1e-3, bvals=(0.0,))
    p.TE = 1000.0
    S, h = oracle.run(p, return_history=True)
    assert np.abs(h - 8000.0).max() < 1e-11 * 8000.0


def test_conjugate_symmetry_and_real_echo():
    """S(t_n; -g) = conj(S(t_n; g)) at every step (real data), and for the
    symmetric PGSE pair the echo signal at TE is real: the product of the
    complex-symmetric step operators is palindromic up to conjugation (P-3)."""
    p = geom.cfg2(n=5, kappa=1e-4, bvals=(3000.0,))
    p.D_cmpt = np.array([2e-3, 1e-3])
    p.dirs = np.array([[0.6, 0.8, 0.0], [-0.6, -0.8, 0.0]])
    p.tet_cmpt = geom.label_sphere(p.xyz, p.tets, np.array([2.0, -1.0, 0.5]), 5.0)
    S, h = oracle.run(p, return_history=True)
    assert np.abs(h[0] - np.conj(h[1])).max() < 1e-12 * abs(h[0, 0])
    assert np.abs(h[0].imag).max() > 1e-4 * abs(h[0, 0])     # genuinely complex midway
    assert abs(S[0].imag) < 1e-12 * abs(S[0])


def test_phase_sign_without_diffusion():
    """D = 0: U(x, t) = exp(-i q F(t) qhat.x) (Eq. strong_BT).  The discrete
    solution refocuses exactly at TE, and at t = delta the nodal phase follows
    -q F x."""
    p = geom.cfg1(n=12)
    p.D_cmpt = np.array([0.0])
    p.bvals = np.array([50.0])
    a = bo.assemble(p)
    S, h = oracle.run_lab(p, a, return_history=True)
    assert abs(h[0, -1] - 64000.0) < 1e-10 * 64000.0
    import scipy.sparse.linalg as spla
    q = float(oracle.q_from_b(50.0, p.delta, p.Delta))
    _, F = oracle.pgse_tables(p.delta, p.Delta, p.dt, p.n_steps)
    L = (a["M"] + 0.5 * p.dt * 1j * q * a["Mx"]).tocsc()
    R = a["M"] - 0.5 * p.dt * 1j * q * a["Mx"]
    lu = spla.splu(L)
    u = np.ones(a["n"], complex)
    for n in range(50):
        u = lu.solve(R @ u)
    x = p.xyz[a["dof_node"], 0]
    err = np.abs(np.angle(u * np.exp(1j * q * F[50] * x)))
    assert q * F[50] * 20.0 > 1.0 and err.max() < 0.05, err.max()


def test_free_periodic_exact_discrete_closed_form():
    """Periodic box, no compartments, transformed frame: u stays spatially
    constant and S/|Omega| = prod_n (1 - (1-th) dt D q^2 F_{n-1}^2) /
    (1 + th dt D q^2 F_n^2) exactly, which tends to exp(-bD) (P-5)."""
    p = geom.free_periodic_box(n=5, L=8.0, dirs=((0.3, 0.4, np.sqrt(0.75)),), bvals=(2000.0,))
    S = oracle.run(p)[0] / 512.0
    q = float(oracle.q_from_b(2000.0, p.delta, p.Delta))
    _, F = oracle.pgse_tables(p.delta, p.Delta, p.dt, p.n_steps)
    D, th, dt = 2e-3, 0.5, p.dt
    prod = np.prod((1 - (1 - th) * dt * D * q * q * F[:-1] ** 2) / (1 + th * dt * D * q * q * F[1:] ** 2))
    assert abs(S - prod) < 1e-13
    assert abs(prod - math.exp(-2000.0 * D)) < 2e-3 * math.exp(-4.0)


def test_kappa_zero_separates():
    """kappa = 0: the two-compartment signal is the sum of separate runs on the
    inside-only and outside-only meshes (P-6)."""
    p = geom.cfg2(n=6, kappa=0.0, bvals=(1500.0,))
    p.kappa_cmpt = np.array([math.inf, 0.0])
    S = oracle.run(p)[0]
    parts = 0.0
    for c in (0, 1):
        q = copy.copy(p)
        keep = p.tet_cmpt == c
        q.tets = p.tets[keep]
        q.tet_cmpt = p.tet_cmpt[keep]
        parts += oracle.run(q)[0]
    assert abs(S - parts) < 1e-12 * abs(S)


def test_large_kappa_limit_is_first_order():
    """Large kappa: difference from the undoubled single-compartment run on the
    same mesh decays like 1/kappa (P-7)."""
    base = geom.cfg2(n=6, bvals=(2000.0,))
    one = copy.copy(base)
    one.tet_cmpt = np.zeros_like(base.tet_cmpt)
    one.D_cmpt = base.D_cmpt[:1]
    one.kappa_cmpt = base.kappa_cmpt[:1]
    S1 = oracle.run(one)[0]
    errs = []
    for k in [1e-2, 1e-1, 1.0]:
        q = copy.copy(base)
        q.kappa_cmpt = np.array([math.inf, k])
        errs.append(abs(oracle.run(q)[0] - S1))
    slopes = np.diff(np.log10(errs))
    assert np.all(np.abs(slopes + 1.0) < 0.1), slopes


def test_axis_permutation_symmetry():
    """A centred sphere on the Kuhn grid: S(x) = S(y) = S(z) (P-8)."""
    p = geom.cfg2(n=6, kappa=1e-4, bvals=(2500.0,))
    p.dirs = np.eye(3)
    S = oracle.run(p)
    assert np.abs(S - S[0]).max() < 1e-12 * abs(S[0])


def test_lab_converges_to_matrix_formalism_second_order():
    """Slab with the 1-D matrix-formalism limit; h and dt halved together:
    errors shrink by about 4 per halving (P-4, P-9)."""
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    ref = oracle.mf_interval_signal(40.0, 2e-3, q, 2500.0, 5000.0, 400).real
    errs = []
    for nx, dt in [(48, 50.0), (96, 25.0), (192, 12.5)]:
        p = geom.slab_1d(nx, dt=dt)
        S = oracle.run(p)[0] / 40.0
        errs.append(abs(S.real - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_transformed_frame_agrees_with_lab_in_neumann_box():
    """Both frames discretise the same PDE; on a Neumann box with a permeable
    sphere they agree to discretisation error, which shrinks with h and dt."""
    diffs = []
    for n, dt in [(6, 100.0), (12, 50.0)]:
        p = geom.cfg2(n=n, dt=dt, kappa=1e-4, bvals=(2000.0,))
        a = bo.assemble(p)
        Sl = oracle.run_lab(p, a)[0]
        St = oracle.run_transformed(p, a)[0]
        diffs.append(abs(Sl - St) / abs(Sl))
    assert diffs[1] < 0.15 and diffs[1] < diffs[0] / 2.0, diffs


def test_direct_and_iterative_routes_agree():
    """The ILU-preconditioned Krylov route (used above a few thousand unknowns)
    reproduces the sparse-LU route to rounding, in both frames."""
    p = geom.cfg2(n=6, kappa=1e-4, bvals=(1000.0, 3000.0))
    a = bo.assemble(p)
    S1 = oracle.run(p, a, route="lu")
    S2 = oracle.run(p, a, route="iter")
    assert np.abs(S1 - S2).max() < 1e-12 * np.abs(S1).max()
    p = geom.cfg3(n=6, n_dir=1, n_b=2)
    a = bo.assemble(p)
    S1 = oracle.run(p, a, route="lu")
    S2 = oracle.run(p, a, route="iter")
    assert np.abs(S1 - S2).max() < 1e-12 * np.abs(S1).max()


def test_direct_and_iterative_routes_agree_at_full_cfg1_size():
    """The stored full-size oracle signals are produced by the iterative route
    (above a few thousand unknowns).  At cfg1's full 15,625 unknowns the sparse
    LU is still affordable: both routes give the same signal to rounding, and
    the stored value with it."""
    import json
    import os
    p = geom.cfg1()
    S_lu = oracle.run(p, route="lu")
    S_it = oracle.run(p, route="iter")
    assert abs(S_lu[0] - S_it[0]) <= 1e-12 * abs(S_lu[0])
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg1_full.json")) as f:
        g = json.load(f)
    assert abs(S_lu[0] - complex(g["S_re"][0], g["S_im"][0])) <= 1e-12 * abs(S_lu[0])


def test_step_average_reading_keeps_second_order():
    """Reading Q1: the theta-scheme with f evaluated at the step ends (the
    literal form) integrates the PGSE lobes by the trapezoid rule, which gives
    the first lobe delta + dt/2 and the second -delta: a net phase q dt/2 at TE.
    On a fibre whose gradient origin is off its centre that phase shows up as
    a first-order error with a spurious imaginary part, while the step
    averages (F(TE) = 0 exactly) stay second order with a real signal.  The
    literal stepping is written out here only to show the defect."""
    import scipy.sparse.linalg as spla
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))

    def f_point(t):
        return 1.0 if 0.0 <= t <= 2500.0 else (-1.0 if 5000.0 < t <= 7500.0 else 0.0)

    def fibre(dt):
        p = geom.line_segments(96, dt=dt)
        p.box_lo, p.box_hi = np.array([-20.0, -20.0, -20.0]), np.array([60.0, 20.0, 20.0])
        return p

    def literal(p):
        a = bo.assemble(p)
        M, K, Mx = a["M"].tocsc(), a["K"].tocsc(), a["Mx"].tocsc()
        u = np.ones(a["n"], complex)
        for k in range(1, p.n_steps + 1):
            fn, fo = f_point(k * p.dt), f_point((k - 1) * p.dt)
            u = spla.spsolve((M + 0.5 * p.dt * (K + 1j * q * fn * Mx)).tocsc(),
                             (M - 0.5 * p.dt * (K + 1j * q * fo * Mx)) @ u)
        return (a["M"] @ np.ones(a["n"])) @ u / 40.0

    ref = oracle.run(fibre(3.125))[0] / 40.0
    lit, avg = [], []
    for dt in (50.0, 25.0, 12.5):
        Sl = literal(fibre(dt))
        Sa = oracle.run(fibre(dt))[0] / 40.0
        lit.append(abs(Sl - ref))
        avg.append(abs(Sa - ref))
        assert abs(Sa.imag) < 1e-12 and abs(Sl.imag) > 2e-4 * dt      # a phase of order dt
        fbar, F, _ = oracle.sequence(fibre(dt))
        assert abs(F[-1]) < 1e-9
    assert 1.7 < lit[0] / lit[1] < 2.3 and 1.7 < lit[1] / lit[2] < 2.3, lit
    assert 3.5 < avg[0] / avg[1] < 4.7 and 3.5 < avg[1] / avg[2] < 4.7, avg


def test_periodic_cylinder_transformed_converges_to_disk_matrix_formalism():
    """3-D tetrahedra of a disk extruded along a periodic z axis (transformed
    frame), gradient across the axis: the signal per volume approaches the
    disk's matrix-formalism value at second order as h and dt halve together
    (a curved boundary, unlike the box pins)."""
    from oracle import mfdisk
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    ref = mfdisk.mf_disk_signal(5.0, 2e-3, q, 2500.0, 5000.0).real
    errs = []
    for m, dt in ((6, 50.0), (12, 25.0), (24, 12.5)):
        p = geom.periodic_cylinder(m, dt=dt, dirs=((0.6, 0.8, 0.0),))
        X = p.xyz[p.tets]
        vol = np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0])).sum() / 6.0
        errs.append(abs(oracle.run(p)[0].real / vol - ref))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs


@pytest.mark.parametrize("maker", [lambda: geom.layered_sphere(n=8, bvals=(0.0,)),
                                   lambda: geom.layered_torus(h=4.0, bvals=(0.0,))])
def test_three_layer_structures_conserve_at_zero_gradient(maker):
    """Section 4's three-layer sphere and torus, layers of different D with
    permeable membranes: at g = 0 the signal stays the volume at every step."""
    p = maker()
    p.dt, p.delta, p.Delta, p.TE = 50.0, 1000.0, 2000.0, 3000.0
    X = p.xyz[p.tets]
    vol = np.abs(np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))).sum() / 6
    S, H = oracle.run(p, return_history=True)
    assert np.max(np.abs(H[0] - vol)) < 1e-10 * vol


def test_stored_signals_still_match_the_oracle():
    """The stored oracle signals the GPU tests read must still be what the
    oracle computes (cheapest stored case, every RHS, with its fingerprint)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg2_n12_dt100.json")
    g = json.load(open(path))
    p = geom.cfg2(**g["kwargs"])
    assert len(p.xyz) == g["fingerprint"]["n_nodes"] and len(p.tets) == g["fingerprint"]["n_tets"]
    S = oracle.run(p, rhs=g["rhs"])
    ref = np.array(g["S_re"]) + 1j * np.array(g["S_im"])
    assert np.max(np.abs(S - ref) / np.abs(ref)) < 1e-12

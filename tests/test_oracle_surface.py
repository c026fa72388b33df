"""Pins of the thin-layer discretisation: P1 triangles of a surface embedded
in 3-D with tangential gradients.  A rotated planar mesh must reproduce the
planar family exactly (the 2-D pins then carry over); on the sphere, the
generalized eigenvalues of (K, M) must converge at second order to the
Laplace-Beltrami eigenvalues D l(l+1)/R^2; a membrane along a circle of
latitude must carry kappa times its length; the total area is conserved at
g = 0."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import geom
import oracle
from oracle import btoracle as bo


def _rotation():
    a, b, c = 0.7, -0.4, 1.1
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    Ry = np.array([[math.cos(c), 0, math.sin(c)], [0, 1, 0], [-math.sin(c), 0, math.cos(c)]])
    return Rz @ Rx @ Ry


def test_rotated_plane_reproduces_the_planar_family():
    p = geom.square_disk(n=10, L=10.0, R=3.0, kappa=1e-4, bvals=(1000.0, 3000.0), dirs=((0.6, 0.8, 0.0),))
    Q = _rotation()
    s = geom.square_disk(n=10, L=10.0, R=3.0, kappa=1e-4, bvals=(1000.0, 3000.0),
                         dirs=(Q @ np.array([0.6, 0.8, 0.0]),))
    s.xyz = p.xyz @ Q.T
    s.surface = True
    s.box_lo, s.box_hi = np.full(3, -6.0), np.full(3, 6.0)       # same centre (the origin)
    a, b = bo.assemble(p), bo.assemble(s)
    for nm in ("M", "K", "J", "MD"):
        scale = abs(a[nm]).max()
        assert abs(a[nm] - b[nm]).max() < 1e-13 * scale, nm
    Mp = [a["Mx"], a["My"], a["Mz"]]
    for k, nm in enumerate(("Mx", "My", "Mz")):
        want = sum(Q[k, l] * Mp[l] for l in range(3))
        assert abs(b[nm] - want).max() < 1e-12 * abs(a["Mx"]).max(), nm
    Sp, Ss = oracle.run(p), oracle.run(s)
    assert np.max(np.abs(Sp - Ss) / np.abs(Sp)) < 1e-11


def _lb_eigs(level, R=2.0):
    p = geom.spherical_shell(level=level, R=R, D=1.0)
    a = bo.assemble(p)
    w = sla.eigh(a["K"].toarray(), a["M"].toarray(), eigvals_only=True, subset_by_index=[0, 15])
    return w


def test_sphere_laplace_beltrami_eigenvalues_second_order():
    """Eigenvalues 0 (once), 2/R^2 (three times), 6/R^2 (five), 12/R^2 (seven)."""
    R = 2.0
    exact = np.repeat([0.0, 2.0, 6.0, 12.0], [1, 3, 5, 7]) / R ** 2
    errs = []
    for level in (2, 3, 4):
        w = _lb_eigs(level, R)
        assert abs(w[0]) < 1e-10
        errs.append(np.max(np.abs(w[1:] - exact[1:]) / exact[1:]))
    assert errs[2] < 6e-3
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs


@pytest.fixture(scope="module")
def capped():
    p = geom.spherical_shell(level=3, R=5.0, kappa=1e-4, cap_z=0.3)
    return p, bo.assemble(p)


def test_membrane_along_latitude_carries_kappa_times_length(capped):
    p, a = capped
    edges = {}
    for t, tri in enumerate(p.tets):
        for e in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
            edges.setdefault(tuple(sorted(e)), []).append(p.tet_cmpt[t])
    length = sum(np.linalg.norm(p.xyz[i] - p.xyz[j]) for (i, j), c in edges.items() if len(c) == 2 and c[0] != c[1])
    assert length > 0
    side = (a["dof_cmpt"] == 1).astype(float)
    assert abs(-(side @ a["J"] @ (1 - side)) - 1e-4 * length) < 1e-14 * length
    # areas: 1^T M 1 is the surface area of the triangles
    X = p.xyz[p.tets]
    area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1).sum()
    one = np.ones(a["n"])
    assert abs(one @ a["M"] @ one - area) < 1e-12 * area
    for nm in ("K", "J"):
        assert np.abs(a[nm] @ one).max() < 1e-14


def test_shell_conserves_at_zero_gradient_and_conjugates(capped):
    p, a = capped
    X = p.xyz[p.tets]
    area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1).sum()
    q = geom.spherical_shell(level=3, R=5.0, kappa=1e-4, cap_z=0.3, bvals=(0.0,))
    S, H = oracle.run(q, return_history=True)
    assert np.max(np.abs(H[0] - area)) < 1e-10 * area
    d = np.array([0.3, -0.5, 0.8])
    s1 = geom.spherical_shell(level=2, R=5.0, kappa=1e-4, cap_z=0.3, bvals=(2000.0,), dirs=(d,))
    s2 = geom.spherical_shell(level=2, R=5.0, kappa=1e-4, cap_z=0.3, bvals=(2000.0,), dirs=(-d,))
    a1, a2 = oracle.run(s1)[0], oracle.run(s2)[0]
    assert abs(a1 - np.conj(a2)) < 1e-12 * abs(a1)


def test_surface_refusals():
    p = geom.spherical_shell(level=1)
    p.transformed = True
    with pytest.raises(ValueError):
        bo.assemble(p)


def test_shell_matrix_formalism_limits():
    """Diffusion on a spherical shell: the narrow-pulse long-time limit of the
    matrix formalism is [sin(kR) / (kR)]^2, the squared mean of e^{ikz} over the
    sphere; no gradient leaves 1; truncation converges."""
    from oracle import mfshell
    R = 5.0
    for k in (0.3, 0.8):
        s = mfshell.mf_shell_signal(R, 2e-3, k, 1.0, 2e6)
        want = (math.sin(k * R) / (k * R)) ** 2
        assert abs(s - want) < 2e-3 * want, (k, s, want)
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    assert abs(mfshell.mf_shell_signal(R, 2e-3, 0.0, 2500.0, 5000.0) - 1.0) < 1e-12
    assert abs(mfshell.mf_shell_signal(R, 2e-3, q, 2500.0, 5000.0, 30) -
               mfshell.mf_shell_signal(R, 2e-3, q, 2500.0, 5000.0, 60)) < 1e-12


def test_icosphere_converges_to_shell_matrix_formalism_second_order():
    """Surface triangles on refined icospheres with dt halved together: the
    signal per area approaches the shell's matrix-formalism value at second
    order (error ratios about 4)."""
    from oracle import mfshell
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    ref = mfshell.mf_shell_signal(5.0, 2e-3, q, 2500.0, 5000.0).real
    errs = []
    for level, dt in ((2, 50.0), (3, 25.0), (4, 12.5)):
        p = geom.spherical_shell(level=level, R=5.0, dt=dt, bvals=(1000.0,), dirs=((0.0, 0.0, 1.0),))
        X = p.xyz[p.tets]
        area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1).sum()
        errs.append(abs(oracle.run(p)[0].real / area - ref))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs

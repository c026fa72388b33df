"""Pins of anisotropic diffusion (one symmetric tensor per compartment in
div(D grad U), Section 2).  The discrete energy of a linear field u = a.x is
exact for P1 elements: u^T K u = sum_c a^T D_c a |Omega_c| with the volumes
summed from the tetrahedra; six directions a fix all six tensor components
(a swapped or transposed component fails).  Also: K symmetric with K 1 = 0,
and an isotropic tensor reproduces the scalar-D run."""
import numpy as np
import pytest

import geom
import oracle
from oracle import btoracle as bo


def _volumes(p):
    X = p.xyz[p.tets]
    v = np.abs(np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))) / 6.0
    return np.bincount(p.tet_cmpt, weights=v, minlength=p.n_cmpt)


def _full(t):
    xx, yy, zz, xy, yz, zx = t
    return np.array([[xx, xy, zx], [xy, yy, yz], [zx, yz, zz]])


TENSORS = np.array([[2.0e-3, 1.1e-3, 0.6e-3, 0.3e-3, -0.2e-3, 0.15e-3],
                    [1.0e-3, 1.5e-3, 2.5e-3, -0.4e-3, 0.35e-3, 0.1e-3]])


@pytest.mark.parametrize("a", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1), (0.3, -0.7, 0.5)])
def test_linear_field_energy_is_exact(a):
    p = geom.cfg2(n=5, kappa=1e-4)
    p.D_tensor = TENSORS
    asm = bo.assemble(p)
    K = asm["K"]
    a = np.asarray(a, float)
    u = p.xyz[asm["dof_node"]] @ a
    vol = _volumes(p)
    want = sum(vol[c] * a @ _full(TENSORS[c]) @ a for c in range(p.n_cmpt))
    assert abs(u @ (K @ u) - want) < 1e-12 * abs(want)


def test_tensor_stiffness_symmetric_and_annihilates_constants():
    p = geom.cfg2(n=5, kappa=1e-4)
    p.D_tensor = TENSORS
    K = bo.assemble(p)["K"]
    scale = abs(K).max()
    assert abs(K - K.T).max() < 1e-14 * scale       # equal up to rounding order
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13 * scale


def test_isotropic_tensor_equals_scalar_run():
    p = geom.cfg2(n=5, kappa=1e-4, bvals=(1500.0,))
    ref = oracle.run(p)
    p.D_tensor = np.array([[d, d, d, 0.0, 0.0, 0.0] for d in p.D_cmpt])
    assert np.max(np.abs(oracle.run(p) - ref)) < 1e-12 * np.max(np.abs(ref))


# ---------------------------------------------------------------- cell-based tensors
def _random_spd(n, rng):
    A = rng.normal(size=(n, 3, 3)) * 1e-2
    S = np.einsum("nij,nkj->nik", A, A) + 1e-4 * np.eye(3)[None]
    return np.stack([S[:, 0, 0], S[:, 1, 1], S[:, 2, 2], S[:, 0, 1], S[:, 1, 2], S[:, 2, 0]], axis=1)


def test_element_tensors_linear_field_energy_is_exact():
    """With one tensor per element, u^T K u = sum_e |T_e| a^T D_e a for every
    linear field u = a.x (each element's own tensor, no compartment lookup)."""
    rng = np.random.default_rng(7)
    p = geom.cfg2(n=5, kappa=1e-4)
    p.D_tensor_elem = _random_spd(len(p.tets), rng)
    asm = bo.assemble(p)
    X = p.xyz[p.tets]
    vol = np.abs(np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))) / 6.0
    for a in ([1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1], [1, 0, 1], [0.3, -0.7, 0.5]):
        a = np.asarray(a, float)
        u = p.xyz[asm["dof_node"]] @ a
        want = sum(vol[e] * a @ _full(p.D_tensor_elem[e]) @ a for e in range(len(vol)))
        assert abs(u @ (asm["K"] @ u) - want) < 1e-12 * abs(want)
    assert abs(asm["K"] - asm["K"].T).max() < 1e-15 * abs(asm["K"]).max()


def test_element_tensors_expanding_compartment_tensors_agree():
    p = geom.cfg2(n=5, kappa=1e-4, bvals=(1500.0,))
    p.dirs = np.array([[0.0, 0.6, 0.8]])
    p.D_tensor = TENSORS
    q = geom.cfg2(n=5, kappa=1e-4, bvals=(1500.0,))
    q.dirs = p.dirs
    q.D_tensor_elem = TENSORS[q.tet_cmpt]
    a, b = bo.assemble(p), bo.assemble(q)
    assert abs(a["K"] - b["K"]).max() == 0.0
    assert np.array_equal(oracle.run(p), oracle.run(q))


# ---------------------------------------------------------------- tensors in the transformed frame
def _quad4():
    a, b = 0.5854101966249685, 0.1381966011250105     # 4-point rule, exact for quadratics
    return np.array([[a, b, b, b], [b, a, b, b], [b, b, a, b], [b, b, b, a]])


def test_transformed_tensor_form_equals_gauge_energy():
    """u^H (K + q^2F^2 MD_q + i q F Eq) u = sum_T |T| <(grad u - i qF qhat u)^H D_T
    (grad u - i qF qhat u)> with a rule exact for quadratics, D_T one SPD tensor
    per element: fixes E_k with D grad phi and the qhat^T D qhat mass."""
    rng = np.random.default_rng(3)
    p = geom.cfg2(n=4)
    p.D_tensor_elem = _random_spd(len(p.tets), rng)
    a = bo.assemble(p)
    u = rng.normal(size=a["n"]) + 1j * rng.normal(size=a["n"])
    qh = np.array([0.3, -0.5, 0.81]); qh /= np.linalg.norm(qh)
    qF = 0.37
    xx, yy, zz, xy, yz, zx = a["MDt"]
    MDq = (qh[0] ** 2 * xx + qh[1] ** 2 * yy + qh[2] ** 2 * zz +
           2 * (qh[0] * qh[1] * xy + qh[1] * qh[2] * yz + qh[2] * qh[0] * zx))
    Eq = qh[0] * a["Ex"] + qh[1] * a["Ey"] + qh[2] * a["Ez"]
    lhs = np.vdot(u, (a["K"] + qF * qF * MDq + 1j * qF * Eq) @ u)
    X = p.xyz[p.tets]
    vol, G = bo.tet_geometry(X)
    ue = u[a["tet_dof"]]
    g = np.einsum("ti,tik->tk", ue, G)
    uq = ue @ _quad4().T
    v = g[:, None, :] - 1j * qF * qh[None, None, :] * uq[:, :, None]          # [nt, 4, 3]
    Dm = np.array([_full(t) for t in p.D_tensor_elem])
    dens = np.einsum("tqk,tkl,tql->tq", np.conj(v), Dm, v).real
    rhs = np.sum(vol * 0.25 * dens.sum(axis=1))
    assert abs(lhs.imag) < 1e-12 * abs(rhs)
    assert abs(lhs.real - rhs) < 1e-12 * abs(rhs)


def test_periodic_anisotropic_free_diffusion_exact_product():
    """Free diffusion with one tensor D in a periodic box, transformed frame:
    u stays constant and S/|Omega| = prod (1 - (1-th) dt Dq q^2 F_{n-1}^2) /
    (1 + th dt Dq q^2 F_n^2) with Dq = qhat^T D qhat (P-5 with a tensor)."""
    D6 = np.array([2.0e-3, 1.1e-3, 0.6e-3, 0.3e-3, -0.2e-3, 0.15e-3])
    for qh in ([1.0, 0.0, 0.0], [0.3, 0.4, np.sqrt(0.75)], [0.0, 0.6, -0.8]):
        p = geom.free_periodic_box(n=4, L=6.0, dirs=(qh,), bvals=(1500.0,))
        p.D_tensor = D6[None, :]
        S = oracle.run(p)[0] / 216.0
        qv = np.asarray(qh)
        Dq = qv @ _full(D6) @ qv
        _, F, I = oracle.sequence(p)
        q2 = 1500.0 / I
        prod = np.prod((1 - 0.5 * p.dt * Dq * q2 * F[:-1] ** 2) / (1 + 0.5 * p.dt * Dq * q2 * F[1:] ** 2))
        assert abs(S - prod) < 1e-12, (qh, S, prod)


def test_transformed_isotropic_tensor_reproduces_scalar_run():
    p = geom.cfg3(n=6, n_dir=2, n_b=1)
    ref = oracle.run(p)
    p.D_tensor = np.array([[d, d, d, 0.0, 0.0, 0.0] for d in p.D_cmpt])
    assert np.max(np.abs(oracle.run(p) - ref) / np.abs(ref)) < 1e-12


def test_lab_and_transformed_frames_agree_with_tensors():
    """Both frames discretise the same PDE; with per-element tensors in a
    Neumann box with a permeable sphere their gap shrinks at second order as h
    and dt halve together (0.91 -> 0.21 here: the coarse lab frame is far off)."""
    gaps = []
    for n, dt in ((6, 100.0), (12, 50.0)):
        p = geom.cfg2(n=n, dt=dt, kappa=1e-4, bvals=(2000.0,))
        p.dirs = np.array([[0.0, 0.6, 0.8]])
        p.D_tensor = TENSORS
        lab = oracle.run(p)[0]
        p.transformed = True
        tr = oracle.run(p)[0]
        gaps.append(abs(lab - tr) / abs(lab))
    assert gaps[0] / gaps[1] > 3.0, gaps

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


def test_element_tensors_refused_in_transformed_frame():
    p = geom.free_periodic_box(n=3, L=5.0)
    p.D_tensor_elem = np.tile([2e-3, 2e-3, 2e-3, 0, 0, 0], (len(p.tets), 1))
    with pytest.raises(ValueError):
        oracle.run(p)

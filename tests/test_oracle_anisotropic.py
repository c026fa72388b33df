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

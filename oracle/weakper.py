"""Oracle side of the weak pseudo-periodic boundary conditions (Appendix B,
"Weak implementation of the pseudo-periodic BCs").  TEST INFRASTRUCTURE ONLY.

On a box that is not meshed periodically, the faces x_k = lo_k (master) and
x_k = hi_k (slave) are coupled through an artificial permeability kappa_e:
  D grad U_m . n_m = kappa_e (U_s e^{i theta_ms} - U_m),
  D grad U_s . n_s = kappa_e (U_m e^{i theta_sm} - U_s),
  theta_ms = -theta_sm = gamma g . (x_s - x_m) F(t) = q qhat_k L_k F(t),
with U_s taken at the previous time step (operator splitting of Appendix B).
In matrix form, with B the boundary-face mass on both sides and C_n the
face-mass coupling of each face with its partner face times e^{+-i theta^n}:
  L_n = M + th dt (A_n + kappa_e B),  rhs = R_n u^{n-1} + th dt kappa_e C_n u^{n-1}.
Appendix B weighs the implicit part by theta and the explicit part by
(1 - theta); both are weighted by theta here (equal at theta = 1/2, and
consistent for every theta).  The partner face is found by shifting the
master face by L_k along axis k: the mesh must match across the box.
kappa_e defaults to max_c D_c / h (the paper's Nitsche-consistent choice) with
h = (d! x mean element measure)^(1/d), the Kuhn cell edge in d = 3 or 2.
In 2-D (triangles in the xy plane) the faces are boundary edges and only the
x and y axes can be coupled.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

_LOC = {4: np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]),
        3: np.array([[1, 2], [0, 2], [0, 1]])}


def default_kappa_e(p, vol):
    d = p.tets.shape[1] - 1
    h = (math.factorial(d) * float(np.mean(vol))) ** (1.0 / d)
    return float(np.max(p.D_cmpt)) / h


def box_faces(p, axes):
    """Boundary faces on the selected box sides: list of (element, local
    vertex indices of the face, axis, side) with side 0 = lo (master), 1 = hi
    (slave)."""
    nv = p.tets.shape[1]
    if getattr(p, "surface", False):
        raise ValueError("a surface has no box sides to couple")
    if nv not in _LOC or (nv == 3 and axes & 4):
        raise ValueError("weak periodic faces need tetrahedra, or triangles coupled along x and y")
    loc = _LOC[nv]
    lo, hi = np.asarray(p.box_lo, float), np.asarray(p.box_hi, float)
    tol = 1e-9 * float(np.max(hi - lo))
    out = []
    X = p.xyz[p.tets]                                   # [nt, nv, 3]
    for k in range(3):
        if not (axes >> k) & 1:
            continue
        for side, plane in ((0, lo[k]), (1, hi[k])):
            on = np.abs(X[:, :, k] - plane) < tol      # [nt, nv]
            for f in range(nv):
                t = np.flatnonzero(np.all(on[:, loc[f]], axis=1))
                out += [(int(ti), loc[f], k, side) for ti in t]
    return out


def face_mass(Xf):
    """P1 mass of a boundary face: a triangle, area / 12 (1 + delta_ab), or an
    edge, length / 6 (1 + delta_ab)."""
    fs = len(Xf)
    if fs == 3:
        meas = 0.5 * np.linalg.norm(np.cross(Xf[1] - Xf[0], Xf[2] - Xf[0]))
    else:
        meas = np.linalg.norm(Xf[1] - Xf[0])
    return meas / (fs * (fs + 1)) * (np.ones((fs, fs)) + np.eye(fs))


def operators(p, asm, axes, kappa_e=None):
    """(B, pairs, kappa_e, L): B [n, n] boundary mass, pairs = list of
    (row dof, col dof, weight, axis, sign) for the coupling C."""
    X = p.xyz[p.tets]
    if p.tets.shape[1] == 4:
        vol = np.abs(np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))) / 6.0
    else:
        vol = 0.5 * np.abs(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])[:, 2])
    ke = default_kappa_e(p, vol) if kappa_e is None else float(kappa_e)
    L = np.asarray(p.box_hi, float) - np.asarray(p.box_lo, float)
    tol = 1e-9 * float(np.max(L))
    n = asm["n"]
    tet_dof = asm["tet_dof"]
    faces = box_faces(p, axes)
    rows, cols, vals = [], [], []
    # slave faces by axis: key = sorted quantized coordinates of the nodes moved to the lo side
    index = {}
    for (t, lf, k, side) in faces:
        Xf = p.xyz[p.tets[t, lf]]
        dofs = tet_dof[t, lf]
        Mf = face_mass(Xf)
        fs = len(lf)
        for a in range(fs):
            for b in range(fs):
                rows.append(dofs[a]), cols.append(dofs[b]), vals.append(Mf[a, b])
        if side == 1:
            Xm = Xf.copy()
            Xm[:, k] -= L[k]
            key = (k, tuple(sorted(tuple(np.round(x / tol).astype(np.int64)) for x in Xm)))
            index[key] = (t, lf)
    B = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    pairs = []
    for (t, lf, k, side) in faces:
        if side != 0:
            continue
        Xf = p.xyz[p.tets[t, lf]]
        key = (k, tuple(sorted(tuple(np.round(x / tol).astype(np.int64)) for x in Xf)))
        if key not in index:
            raise ValueError(f"mesh does not match across the box on axis {k}")
        ts, lfs = index[key]
        Xs = p.xyz[p.tets[ts, lfs]]
        # partner of master vertex a: the slave vertex at x_a + L_k e_k
        fs = len(lf)
        perm = []
        for a in range(fs):
            target = Xf[a].copy()
            target[k] += L[k]
            perm.append(int(np.argmin(np.linalg.norm(Xs - target, axis=1))))
        dm = tet_dof[t, lf]
        ds = tet_dof[ts, lfs][perm]
        Mf = face_mass(Xf)
        for a in range(fs):
            for b in range(fs):
                pairs.append((int(dm[a]), int(ds[b]), Mf[a, b], k, +1))   # master row, slave value
                pairs.append((int(ds[a]), int(dm[b]), Mf[a, b], k, -1))   # slave row, master value
    return B, pairs, ke, L


def coupling(pairs, n, q, qhat, L, F):
    """C_n for one RHS at F = F(t_n): sum of weight e^{i sign q qhat_k L_k F}."""
    r = np.array([pp[0] for pp in pairs])
    c = np.array([pp[1] for pp in pairs])
    w = np.array([pp[2] for pp in pairs])
    k = np.array([pp[3] for pp in pairs])
    s = np.array([pp[4] for pp in pairs])
    phase = np.exp(1j * s * q * np.asarray(qhat)[k] * L[k] * F)
    return sp.coo_matrix((w * phase, (r, c)), shape=(n, n)).tocsr()

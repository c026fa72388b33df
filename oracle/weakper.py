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
consistent for every theta).  The partner value is the P1 field of the opposite side at the node shifted by
+-L_k along axis k (the master/slave projection), so the sides need not match.
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


def _tangential(p, k):
    """The coordinates along a side of axis k: the other two axes in 3-D, the
    other in-plane axis for a 2-D mesh."""
    if p.tets.shape[1] == 3:
        return [1] if k == 0 else [0]
    return [a for a in range(3) if a != k]


def _locate(side_faces, y, tang):
    """(dofs, barycentric weights) of the face of `side_faces` containing the
    point y, by its tangential coordinates; the face with the largest smallest
    weight wins, so points on shared edges and vertices are found."""
    best = None
    for Xf, dofs, _ in side_faces:
        P = Xf[:, tang]
        z = y[tang]
        if len(tang) == 2:
            T = np.column_stack([P[1] - P[0], P[2] - P[0]])
            l12 = np.linalg.solve(T, z - P[0])
            lam = np.array([1.0 - l12.sum(), l12[0], l12[1]])
        else:
            s = (z[0] - P[0, 0]) / (P[1, 0] - P[0, 0])
            lam = np.array([1.0 - s, s])
        if best is None or lam.min() > best[0]:
            best = (lam.min(), dofs, lam)
    if best is None or best[0] < -1e-9:
        raise ValueError("a node's partner point lies outside the opposite side of the box")
    return best[1], best[2]


def operators(p, asm, axes, kappa_e=None):
    """(B, pairs, kappa_e, L): B [n, n] boundary mass, pairs = list of
    (row dof, col dof, weight, axis, sign) for the coupling C.

    The partner value on the opposite side is the P1 field there, taken at
    the shifted node positions (the master/slave projection of Appendix B):
    with P the interpolation matrix of those points, C = B_side P.  Rows of P
    sum to 1, so C 1 = B 1; on matching sides P is a permutation."""
    X = p.xyz[p.tets]
    if p.tets.shape[1] == 4:
        vol = np.abs(np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))) / 6.0
    else:
        vol = 0.5 * np.abs(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])[:, 2])
    ke = default_kappa_e(p, vol) if kappa_e is None else float(kappa_e)
    L = np.asarray(p.box_hi, float) - np.asarray(p.box_lo, float)
    n = asm["n"]
    tet_dof = asm["tet_dof"]
    faces = box_faces(p, axes)
    rows, cols, vals = [], [], []
    sides = {}
    for (t, lf, k, side) in faces:
        Xf = p.xyz[p.tets[t, lf]]
        dofs = tet_dof[t, lf]
        Mf = face_mass(Xf)
        fs = len(lf)
        for a in range(fs):
            for b in range(fs):
                rows.append(dofs[a]), cols.append(dofs[b]), vals.append(Mf[a, b])
        sides.setdefault((k, side), []).append((Xf, dofs, Mf))
    B = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    pairs = []
    for k in range(3):
        if not (axes >> k) & 1:
            continue
        tang = _tangential(p, k)
        for side, other, shift, sign in ((0, 1, +L[k], +1), (1, 0, -L[k], -1)):
            partner = {}
            for Xf, dofs, Mf in sides.get((k, side), []):
                for b in range(len(dofs)):
                    if dofs[b] not in partner:
                        y = Xf[b].copy()
                        y[k] += shift
                        partner[dofs[b]] = _locate(sides.get((k, other), []), y, tang)
                for a in range(len(dofs)):
                    for b in range(len(dofs)):
                        pd, pw = partner[dofs[b]]
                        for d, wgt in zip(pd, pw):
                            if wgt != 0.0:
                                pairs.append((int(dofs[a]), int(d), Mf[a, b] * wgt, k, sign))
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

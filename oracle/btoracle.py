"""Plain, slow FP64 CPU finite-element solve of the multi-compartment
Bloch-Torrey equation (test infrastructure only; see the package docstring).

What it follows (section / equation of arXiv 1908.01719):
  * model: Bloch-Torrey PDE (Eq. strong_BT, Section 2) with the T2 term
    (p.inv_T2, default none) and per-compartment initial values (p.rho), the
    permeable interface conditions (Eq. btpde_ic), PGSE profile (Eq. pgse),
    signal S = integral of U at TE (Eq. signal), b-value (Eq. b_value);
  * PUFEM interface treatment (Appendix A): one nodal copy per compartment on
    interface nodes, with the jump term kappa <[u], [v]> on interface faces;
  * theta-method in time and the matrix form A U^n = F (Appendix B,
    Eqs. theta_discretization2, linear_billinear2, matrix_form);
  * strong pseudo-periodic conditions through the gauge transform
    u = U exp(i gamma F(t) g.x) (Appendix A, Eqs. trBlo, Periodic,
    Binterface2 and the weak form F(u, v, t));
  * elements: P1 tetrahedra, P1 triangles for 2-D domains, and, for the
    thin-layer and thin-tube media of the manifold route (Section 1's feature
    list; Section 5, "Realistic neurons"), P1 triangles of a surface and P1
    segments of a curve embedded in 3-D: integrals over the manifold,
    tangential gradients, uniform thickness or cross-section;
  * a diffusion tensor per compartment (p.D_tensor) or per cell
    (p.D_tensor_elem), Section 3 "Diffusion coefficients and tensors", in the
    stiffness, lab frame;
  * temporal profiles other than PGSE integrated from f (oracle/profiles.py,
    Section 3 "General diffusion-encoding sequence");
  * weak pseudo-periodic conditions through an artificial permeability
    (oracle/weakper.py, Appendix B).

Readings where the paper leaves a choice (each is also listed in the design
notes of the repository):
  * f(t) enters each theta step as its average over the step, f_bar_n, on both
    sides of the step (the paper evaluates f at t^n and t^{n-1}, which is
    ambiguous where the PGSE profile jumps exactly at a grid time);
  * the first-moment matrices use coordinates relative to the box centre;
  * a face between compartments a and b has permeability
    1/(1/kappa_a + 1/kappa_b) (an infinite kappa means "no membrane");
  * consistent mass, exact integration;
  * in the transformed frame the interface and Neumann terms combine with the
    volume term into E_k = C_k - C_k^T, C_k[i, j] = D * integral(phi_i d_k phi_j),
    so the step operator is K + J + D q^2 F^2 M + i q F sum_k qhat_k E_k.

Every linear solve is a sparse direct LU (scipy.sparse.linalg.splu), one
factorisation per distinct step matrix, or, above a few thousand unknowns where
3-D fill makes LU impractical, an ILU-preconditioned GMRES/CG solve to a
relative residual of 1e-14 (checked against the LU route in the CPU tests).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# --------------------------------------------------------------------------
# Periodic identification and interface-node doubling (PUFEM, Appendix A)
# --------------------------------------------------------------------------
def periodic_master(xyz, periodic_mask, lo, hi):
    """Map every node to its master node: on a periodic axis k, a node with
    x_k = hi_k is the same unknown as the node with x_k = lo_k and equal other
    coordinates (master-slave periodicity, Section 2, Eq. btpde_bc)."""
    n = len(xyz)
    if periodic_mask == 0:
        return np.arange(n)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    tol = 1e-9 * float(np.max(hi - lo))
    canon = xyz.copy()
    for k in range(3):
        if periodic_mask >> k & 1:
            on_hi = np.abs(canon[:, k] - hi[k]) < tol
            canon[on_hi, k] = lo[k]
    key = np.round(canon / tol).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    # master = smallest node index among identified nodes
    grp_min = np.full(len(first), n, dtype=np.int64)
    np.minimum.at(grp_min, inv.ravel(), np.arange(n))
    return grp_min[inv.ravel()]


def doubling(master, tets, tet_cmpt, n_cmpt):
    """One degree of freedom per (master node, compartment) pair that occurs in
    some tetrahedron of that compartment.  Dofs are numbered in increasing
    (node, compartment) order."""
    keys = master[tets].astype(np.int64) * n_cmpt + tet_cmpt[:, None].astype(np.int64)
    uniq, inv = np.unique(keys.ravel(), return_inverse=True)
    tet_dof = inv.reshape(-1, tets.shape[1])
    return tet_dof, uniq // n_cmpt, uniq % n_cmpt


def interface_faces(master, tets, tet_cmpt):
    """Faces (edges in 2-D) shared by two elements of different compartments.

    Returns (elem_a, elem_b, local vertex indices of the face in elem_a
    [nf, 3] for tetrahedra, [nf, 2] for triangles).  Face keys use master ids, so faces identified by
    periodicity are found too."""
    if tets.shape[1] == 2:                        # 1-D: end points of segments
        loc = np.array([[1], [0]])
    elif tets.shape[1] == 3:                      # 2-D: edges of triangles
        loc = np.array([[1, 2], [0, 2], [0, 1]])
    else:
        loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    nf_loc, fsz = loc.shape                        # faces per element, nodes per face
    mt = master[tets]
    fv = mt[:, loc]                                # [nt, nf_loc, fsz]
    fv_sorted = np.sort(fv, axis=2).reshape(-1, fsz)
    owner = np.repeat(np.arange(len(tets)), nf_loc)
    lface = np.tile(np.arange(nf_loc), len(tets))
    order = np.lexsort(fv_sorted.T[::-1])
    fs = fv_sorted[order]
    same = np.all(fs[1:] == fs[:-1], axis=1)
    i0 = np.flatnonzero(same)
    ta, tb = owner[order][i0], owner[order][i0 + 1]
    la = lface[order][i0]
    diff = tet_cmpt[ta] != tet_cmpt[tb]
    ta, tb, la = ta[diff], tb[diff], la[diff]
    return ta, tb, loc[la]


# --------------------------------------------------------------------------
# Element matrices (P1 tetrahedra, exact integration)
# --------------------------------------------------------------------------
def _cubic_moments(d=3):
    """c[i,j,l] = (1/|T|) * integral over a d-simplex T of lambda_i lambda_j
    lambda_l, from the barycentric integration formula alpha! d! / (|alpha| + d)!."""
    nv = d + 1
    c = np.empty((nv, nv, nv))
    for i in range(nv):
        for j in range(nv):
            for l in range(nv):
                a = np.bincount([i, j, l], minlength=nv)
                num = np.prod([math.factorial(x) for x in a]) * math.factorial(d)
                c[i, j, l] = num / math.factorial(3 + d)
    return c


def seg_geometry(X):
    """Lengths [nt] and tangential barycentric gradients [nt, 2, 3] of segments
    X [nt, 2, 3] of a curve in 3-D: lambda_1 grows from 0 to 1 along e = x_1 - x_0,
    so its gradient along the curve is e / |e|^2."""
    e = X[:, 1] - X[:, 0]
    l2 = np.einsum("ij,ij->i", e, e)
    G = np.empty((len(X), 2, 3))
    G[:, 1] = e / l2[:, None]
    G[:, 0] = -G[:, 1]
    return np.sqrt(l2), G


def surf_geometry(X):
    """Areas [nt] and tangential barycentric gradients [nt, 3, 3] of triangles
    X [nt, 3, 3] anywhere in 3-D (a thin layer as a 2-D manifold).  With the
    edge matrix E (rows x_1 - x_0, x_2 - x_0), grad lambda_1, grad lambda_2 are
    the tangent vectors g with E g = e_a, i.e. the columns of the
    pseudo-inverse E^T (E E^T)^-1; |T| = sqrt(det(E E^T)) / 2."""
    E = X[:, 1:, :] - X[:, :1, :]                  # [nt, 2, 3]
    Gram = np.einsum("tak,tbk->tab", E, E)
    area = 0.5 * np.sqrt(np.linalg.det(Gram))
    P = np.einsum("tak,tab->tkb", E, np.linalg.inv(Gram))   # [nt, 3, 2] pseudo-inverse
    G = np.empty((len(X), 3, 3))
    G[:, 1:, :] = np.transpose(P, (0, 2, 1))
    G[:, 0, :] = -G[:, 1:, :].sum(axis=1)
    return area, G


def tri_geometry(X):
    """Areas [nt] and barycentric gradients [nt, 3, 3] (z = 0) of triangles in the
    xy plane, X [nt, 3, 3]: grad lambda solves E grad = e_a for the edge matrix."""
    E = X[:, 1:, :2] - X[:, :1, :2]                # [nt, 2, 2] edge vectors
    area = 0.5 * np.linalg.det(E)
    Ginv = np.linalg.inv(E)                        # columns: grad lambda_{1,2}
    G = np.zeros((len(X), 3, 3))
    G[:, 1:, :2] = np.transpose(Ginv, (0, 2, 1))
    G[:, 0, :] = -G[:, 1:, :].sum(axis=1)
    return area, G


def tet_geometry(X):
    """Volumes [nt] and barycentric gradients [nt, 4, 3] of tetrahedra X [nt,4,3]."""
    E = X[:, 1:, :] - X[:, :1, :]                 # rows: edge vectors
    vol = np.linalg.det(E) / 6.0
    Ginv = np.linalg.inv(E)                        # columns: grad lambda_{1..3}
    G = np.empty((len(X), 4, 3))
    G[:, 1:, :] = np.transpose(Ginv, (0, 2, 1))
    G[:, 0, :] = -G[:, 1:, :].sum(axis=1)
    return vol, G


def _coo(rows, cols, vals, n):
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(n, n)).tocsr()


def assemble(p):
    """Assemble every matrix of the method for problem `p` (a geom.Problem).

    Returns a dict with the dof map and the CSR matrices
      M   mass                              (Appendix B, matrix M)
      K   stiffness, D-weighted             (Appendix B, matrix S; p.D_tensor gives
                                            one 3x3 tensor per compartment)
      J   interface jump, kappa-weighted    (Appendix B, matrix I)
      Mx, My, Mz  first-moment mass         (Appendix B, matrix J = sum g_k M_k)
      MD  D-weighted mass                   (transformed frame, Appendix A)
      MR  1/T2-weighted mass                (relaxation term of Section 2)
      Ex, Ey, Ez  skew transport matrices   (transformed frame, Appendix A)
    """
    nv = p.tets.shape[1]                           # 4: tetrahedra, 3: triangles, 2: segments
    d = nv - 1
    manifold = nv == 2 or getattr(p, "surface", False)
    if manifold and (p.periodic_mask or p.transformed):
        raise ValueError("manifolds are solved in the lab frame, without periodicity")
    master = periodic_master(p.xyz, p.periodic_mask, p.box_lo, p.box_hi)
    tet_dof, dof_node, dof_cmpt = doubling(master, p.tets, p.tet_cmpt, p.n_cmpt)
    n = len(dof_node)
    if nv == 2 and np.any(dof_node[1:] == dof_node[:-1]):
        raise ValueError("segments of different compartments share a node")
    X = p.xyz[p.tets]                              # unwrapped element coordinates
    if nv == 3 and getattr(p, "surface", False):
        vol, G = surf_geometry(X)
    else:
        vol, G = {4: tet_geometry, 3: tri_geometry, 2: seg_geometry}[nv](X)
    Dt = p.D_cmpt[p.tet_cmpt]
    rows = np.repeat(tet_dof[:, :, None], nv, axis=2)
    cols = np.repeat(tet_dof[:, None, :], nv, axis=1)

    # P1 mass: |T| (1 + delta_ij) / ((d + 1)(d + 2))
    Me = vol[:, None, None] / ((d + 1) * (d + 2)) * (1.0 + np.eye(nv))[None]
    Dten = getattr(p, "D_tensor", None)
    Dten_e = getattr(p, "D_tensor_elem", None)
    De = None
    if Dten is None and Dten_e is None:
        Ke = (Dt * vol)[:, None, None] * np.einsum("tik,tjk->tij", G, G)
    else:
        # anisotropic diffusion: (D grad u, grad v) with one symmetric tensor
        # per compartment, or per cell (Section 3: cell-based piecewise
        # continuous d_jk), given as (xx, yy, zz, xy, yz, zx)
        T = np.asarray(Dten_e if Dten_e is not None else Dten, float)
        Dm = np.empty((len(T), 3, 3))
        Dm[:, 0, 0], Dm[:, 1, 1], Dm[:, 2, 2] = T[:, 0], T[:, 1], T[:, 2]
        Dm[:, 0, 1] = Dm[:, 1, 0] = T[:, 3]
        Dm[:, 1, 2] = Dm[:, 2, 1] = T[:, 4]
        Dm[:, 2, 0] = Dm[:, 0, 2] = T[:, 5]
        De = Dm if Dten_e is not None else Dm[p.tet_cmpt]
        Ke = vol[:, None, None] * np.einsum("tik,tkl,tjl->tij", G, De, G)
    # De: [nt, 3, 3] per-element tensors, or None (isotropic D per compartment)
    centre = 0.5 * (np.asarray(p.box_lo, float) + np.asarray(p.box_hi, float))
    Xc = X - centre
    c3 = _cubic_moments(d)
    out = {"n": n, "tet_dof": tet_dof, "dof_node": dof_node, "dof_cmpt": dof_cmpt,
           "master": master}
    out["M"] = _coo(rows, cols, Me, n)
    out["K"] = _coo(rows, cols, Ke, n)
    out["MD"] = _coo(rows, cols, Dt[:, None, None] * Me, n)
    # relaxation (U/T2, v) of the weak form: mass weighted by 1/T2 per compartment
    invT2 = getattr(p, "inv_T2", None)
    rT2 = np.zeros(len(vol)) if invT2 is None else np.asarray(invT2, float)[p.tet_cmpt]
    out["MR"] = _coo(rows, cols, rT2[:, None, None] * Me, n)
    # the flux of the transformed weak form is D (grad u - i q F qhat u): with a
    # tensor, C_k[i, j] = int phi_i (D grad phi_j)_k and the q^2 F^2 mass is
    # weighted by qhat^T D qhat, kept as six planes MD_ab = sum_e D_e,ab M_e
    DG = G if De is None else np.einsum("tkl,tjl->tjk", De, G)          # [nt, nv, 3]
    Dw = Dt if De is None else np.ones(len(vol))
    for k, nm in enumerate("xyz"):
        Mk = vol[:, None, None] * np.einsum("ijl,tl->tij", c3, Xc[:, :, k])
        out["M" + nm] = _coo(rows, cols, Mk, n)
        Ck = (Dw * vol / (d + 1))[:, None, None] * np.broadcast_to(DG[:, None, :, k], (len(vol), nv, nv))
        out["E" + nm] = _coo(rows, cols, Ck - np.transpose(Ck, (0, 2, 1)), n)
    if De is not None:
        ab = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))
        out["MDt"] = [_coo(rows, cols, De[:, a, b][:, None, None] * Me, n) for a, b in ab]

    # interface jump term kappa <[u], [v]> on faces between compartments
    ta, tb, lv = interface_faces(master, p.tets, p.tet_cmpt)
    nf = len(ta)
    if nf:
        va = p.tets[ta[:, None], lv]                    # global vertices of face (tet a)
        Xa = p.xyz[va]
        if nv == 4:
            area = 0.5 * np.linalg.norm(np.cross(Xa[:, 1] - Xa[:, 0], Xa[:, 2] - Xa[:, 0]), axis=1)
        else:                                           # interface edges: length
            area = np.linalg.norm(Xa[:, 1] - Xa[:, 0], axis=1)
        fs = nv - 1
        ka = p.kappa_cmpt[p.tet_cmpt[ta]]
        kb = p.kappa_cmpt[p.tet_cmpt[tb]]
        with np.errstate(divide="ignore"):
            kap = 1.0 / (1.0 / ka + 1.0 / kb)
        dof_a = tet_dof[ta[:, None], lv]
        # matching vertex on side b, by master id
        mb = master[p.tets[tb]]
        ma = master[va]
        lb = np.argmax(mb[:, None, :] == ma[:, :, None], axis=2)
        dof_b = tet_dof[tb[:, None], lb]
        # face mass of a (d-1)-simplex: |F| (1 + delta_ab) / (d (d + 1))
        Fm = (area * kap)[:, None, None] / (d * (d + 1)) * (1.0 + np.eye(fs))[None]
        d6 = np.concatenate([dof_a, dof_b], axis=1)
        blk = np.block([[np.ones((fs, fs)), -np.ones((fs, fs))], [-np.ones((fs, fs)), np.ones((fs, fs))]])
        F6 = np.tile(Fm, (1, 2, 2)) * blk[None]
        r6 = np.repeat(d6[:, :, None], 2 * fs, axis=2)
        c6 = np.repeat(d6[:, None, :], 2 * fs, axis=1)
        out["J"] = _coo(r6, c6, F6, n)
    else:
        out["J"] = sp.csr_matrix((n, n))
    out["n_iface"] = nf
    out["volume"] = float(vol.sum())
    return out


def initial_field(p, asm):
    """u^0: the initial magnetization rho of each dof's compartment (1 by default)."""
    rho = getattr(p, "rho", None)
    if rho is None:
        return np.ones(asm["n"], dtype=np.complex128)
    return np.asarray(rho, float)[asm["dof_cmpt"]].astype(np.complex128)


def signal_weights(asm):
    """w = M 1: the exact integral of each P1 basis function (Eq. signal)."""
    return asm["M"] @ np.ones(asm["n"])


# --------------------------------------------------------------------------
# Sequence (Eq. pgse, Eq. b_value)
# --------------------------------------------------------------------------
def pgse_f(t, delta, Delta):
    t = np.asarray(t, float)
    return np.where((t >= 0) & (t <= delta), 1.0, np.where((t > Delta) & (t <= Delta + delta), -1.0, 0.0))


def pgse_F(t, delta, Delta):
    """F(t) = integral_0^t f(s) ds for the PGSE profile."""
    t = np.asarray(t, float)
    return np.clip(t, 0.0, delta) - np.clip(t - Delta, 0.0, delta)


def pgse_tables(delta, Delta, dt, n_steps):
    """f_bar[n] (n = 1..N, index n-1) = step average of f over (t_{n-1}, t_n];
    F[n] (n = 0..N) = F(t_n)."""
    t = dt * np.arange(n_steps + 1)
    F = pgse_F(t, delta, Delta)
    fbar = np.diff(F) / dt
    return fbar, F


def sequence(p):
    """(f_bar_n, F_n, int_0^TE F^2) of problem p: PGSE in closed form (Section 2,
    Eq. pgse), or p.profile = {"kind": ..., "n_periods": ..., "ramp": ...}
    integrated numerically from f (oracle/profiles.py).  The time grid
    t_n = n dt of the theta-scheme must end at TE."""
    N = p.n_steps
    if N < 1 or abs(N * p.dt - p.TE) > 1e-9 * p.TE:
        raise ValueError("TE must be a positive integer multiple of dt")
    prof = getattr(p, "profile", None)
    if prof:
        from . import profiles
        return profiles.tables(prof["kind"], p.delta, p.Delta, p.TE, p.dt, prof.get("n_periods", 1),
                               prof.get("ramp"))
    fbar, F = pgse_tables(p.delta, p.Delta, p.dt, N)
    return fbar, F, p.delta * p.delta * (p.Delta - p.delta / 3.0)


def q_from_b(b, delta, Delta):
    """q = gamma |g| from b = q^2 delta^2 (Delta - delta/3) (Eq. b_value with the
    PGSE F(t))."""
    return np.sqrt(np.asarray(b, float) / (delta * delta * (Delta - delta / 3.0)))


# --------------------------------------------------------------------------
# Time stepping (theta-method, Appendix B matrix form)
# --------------------------------------------------------------------------
LU_MAX_DOFS = 6000     # above this, the iterative route (SuperLU fill grows too fast in 3-D)


class _Solver:
    """Solve L x = b for the step matrices of one RHS, caching by a key that
    identifies the matrix.  Two routes, both library primitives:
      * 'lu'  : sparse direct LU (SuperLU, minimum-degree ordering on A^T + A);
      * 'iter': GMRES (complex-symmetric lab matrices) or CG (Hermitian
                positive-definite transformed matrices), preconditioned by an
                incomplete LU of the same matrix, to a relative residual of
                1e-14 (the discrete solution to rounding level).
    A CPU test checks that both routes agree to 1e-12 on the same problem."""

    def __init__(self, n, route=None, hermitian=False):
        self.route = route or ("lu" if n <= LU_MAX_DOFS else "iter")
        self.hermitian = hermitian
        self.cache = {}

    def solve(self, key, build, b, x0=None):
        ent = self.cache.get(key)
        if ent is None:
            A = build().tocsc().astype(np.complex128)
            if self.route == "lu":
                ent = (A, spla.splu(A, permc_spec="MMD_AT_PLUS_A"))
            else:
                ilu = spla.spilu(A, drop_tol=1e-6, fill_factor=30, permc_spec="MMD_AT_PLUS_A")
                P = spla.LinearOperator(A.shape, ilu.solve, dtype=np.complex128)
                ent = (A, P)
            self.cache[key] = ent
        A, f = ent
        if self.route == "lu":
            return f.solve(b)
        nb = np.linalg.norm(b)
        if nb == 0:
            return np.zeros_like(b)
        if self.hermitian:
            x, info = spla.cg(A, b, x0=x0, rtol=1e-14, atol=0.0, M=f, maxiter=2000)
        else:
            x, info = spla.gmres(A, b, x0=x0, rtol=1e-14, atol=0.0, M=f, restart=60, maxiter=200)
        r = np.linalg.norm(b - A @ x) / nb
        if r > 1e-12:
            raise RuntimeError(f"oracle iterative solve stalled at relative residual {r:.2e}")
        return x


def run_lab(p, asm=None, rhs=None, return_history=False, route=None, return_field=False):
    """Lab frame (Neumann outer boundary):
        L_n = M + theta dt (K + J + MR + i q f_bar_n Mq)
        R_n = M - (1 - theta) dt (K + J + MR + i q f_bar_n Mq),  Mq = sum_k qhat_k M_k
        L_n u^n = R_n u^{n-1},  u^0 = rho (1 by default),  S = (M 1)^T u^N."""
    if asm is None:
        asm = assemble(p)
    if p.periodic_mask:
        raise ValueError("periodic boxes need the transformed frame")
    M, KJ = asm["M"], asm["K"] + asm["J"] + asm["MR"]
    w = signal_weights(asm)
    N = p.n_steps
    fbar, Fn, intF2 = sequence(p)
    weak = getattr(p, "weak_periodic", None)
    if weak:
        from . import weakper
        Bw, pairs, ke, Lbox = weakper.operators(p, asm, weak["axes"], weak.get("kappa_e"))
    nb = len(p.bvals)
    rhs = range(p.n_rhs) if rhs is None else rhs
    th, dt = p.theta, p.dt
    out, hist, fields = [], [], []
    for r in rhs:
        qh = p.dirs[r // nb]
        q = math.sqrt(float(p.bvals[r % nb]) / intF2)  # b = q^2 int F^2 (Eq. b_value)
        Mq = qh[0] * asm["Mx"] + qh[1] * asm["My"] + qh[2] * asm["Mz"]
        sol = _Solver(asm["n"], route)
        u = initial_field(p, asm)
        h = [w @ u]
        for n in range(1, N + 1):
            fb = fbar[n - 1]
            A = KJ + (1j * q * fb) * Mq
            rhs = (M - (1.0 - th) * dt * A) @ u
            if weak:
                # artificial permeability on the box faces: implicit own side,
                # partner side from the previous step with the phase of F(t_n)
                rhs = rhs + (th * dt * ke) * (weakper.coupling(pairs, asm["n"], q, qh, Lbox, Fn[n]) @ u)
                u = sol.solve(fb, lambda: M + th * dt * (A + ke * Bw), rhs, x0=u)
            else:
                u = sol.solve(fb, lambda: M + th * dt * A, rhs, x0=u)
            h.append(w @ u)
        out.append(w @ u)
        hist.append(h)
        fields.append(u)
    return _result(np.array(out), hist, fields, return_history, return_field)


def run_transformed(p, asm=None, rhs=None, return_history=False, route=None, return_field=False):
    """Gauge-transformed frame u = U exp(i q F(t) qhat.x) (Appendix A), valid
    for periodic and Neumann outer boundaries:
        A(F) = K + J + q^2 F^2 MD + i q F Eq,  Eq = sum_k qhat_k E_k
        L_n = M + theta dt A(F_n),  R_n = M - (1 - theta) dt A(F_{n-1})
        S = (M 1)^T u^N  (F(TE) = 0 for PGSE, so U = u at TE).
    With diffusion tensors, MD is replaced per direction by
    sum_ab qhat_a qhat_b MD_ab and E_k carries D grad phi (see assemble)."""
    if asm is None:
        asm = assemble(p)
    M, KJ, MD = asm["M"], asm["K"] + asm["J"] + asm["MR"], asm["MD"]
    w = signal_weights(asm)
    N = p.n_steps
    _, F, intF2 = sequence(p)
    if abs(F[-1]) > 1e-12 * max(1.0, p.delta):
        raise ValueError("F(TE) != 0: the signal needs the phase factor")
    nb = len(p.bvals)
    rhs = range(p.n_rhs) if rhs is None else rhs
    th, dt = p.theta, p.dt
    out, hist, fields = [], [], []
    for r in rhs:
        qh = p.dirs[r // nb]
        q = math.sqrt(float(p.bvals[r % nb]) / intF2)  # b = q^2 int F^2 (Eq. b_value)
        Eq = qh[0] * asm["Ex"] + qh[1] * asm["Ey"] + qh[2] * asm["Ez"]
        MDq = MD
        if "MDt" in asm:
            xx, yy, zz, xy, yz, zx = asm["MDt"]
            MDq = (qh[0] ** 2 * xx + qh[1] ** 2 * yy + qh[2] ** 2 * zz +
                   2 * (qh[0] * qh[1] * xy + qh[1] * qh[2] * yz + qh[2] * qh[0] * zx))

        def A(Fv):
            return KJ + (q * q * Fv * Fv) * MDq + (1j * q * Fv) * Eq

        sol = _Solver(asm["n"], route, hermitian=True)
        u = initial_field(p, asm)
        h = [w @ u]
        for n in range(1, N + 1):
            Fn, Fp = F[n], F[n - 1]
            u = sol.solve(Fn, lambda: M + th * dt * A(Fn), (M - (1.0 - th) * dt * A(Fp)) @ u, x0=u)
            h.append(w @ u)
        out.append(w @ u)
        hist.append(h)
        fields.append(u)
    return _result(np.array(out), hist, fields, return_history, return_field)


def _result(out, hist, fields, return_history, return_field):
    """The signals; with return_history also S(t_n) per RHS, with return_field
    also u^N per RHS (rows in the dof numbering of `assemble`)."""
    res = (out,)
    if return_history:
        res += (np.array(hist),)
    if return_field:
        res += (np.array(fields),)
    return res[0] if len(res) == 1 else res


def run(p, asm=None, rhs=None, return_history=False, route=None, return_field=False):
    dn = np.linalg.norm(np.asarray(p.dirs, float), axis=1)
    if np.any(np.abs(dn - 1.0) > 1e-12):
        raise ValueError("gradient directions must be unit vectors (q = gamma |g| carries the magnitude)")
    if p.tets.shape[1] == 3 and not getattr(p, "surface", False) and \
            np.any(np.abs(np.asarray(p.dirs, float)[:, 2]) > 1e-12):
        raise ValueError("2-D meshes need gradient directions in the xy plane")
    f = run_transformed if (p.transformed or p.periodic_mask) else run_lab
    return f(p, asm, rhs, return_history, route, return_field)

"""Seeded synthetic inputs for the diffusion-MRI finite-element solve.

This module builds the *inputs* of the method only: node coordinates, tetrahedra,
the compartment label of each tetrahedron, per-compartment diffusivity and
membrane permeability, the PGSE timing and the gradient directions and b-values.
It holds none of the method's arithmetic (no interface doubling, no element
matrices, no time stepping); both the CPU oracle and the GPU library consume
these arrays independently.

Units follow the paper's own convention (Section 4 uses micrometres and
microseconds): lengths in um, times in us.  With these units D in mm^2/s,
b in s/mm^2 and kappa in m/s keep their numerical values.

Workloads (synthetic stand-ins for the paper's neuron / extracellular meshes,
Section 5, which are not available):
  cfg1  40 um cube, 24^3 Kuhn grid, one compartment, Neumann, 1 RHS
  cfg2  20 um cube, 48^3, centred sphere r = 5 um (two compartments), 5 b-values
  cfg3  30 um periodic box, 64^3, 40 z-cylinders (lognormal radii), 64 dirs x 8 b
  cfg4  40 um cube, 96^3, packed spheres + finite cylinders, 32 dirs x 4 b
  cfg5  32 packings of uneven size (50k .. 2M nodes), 16 dirs x 4 b each
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Background compartment: no membrane of its own.  The permeability of the
# interface between compartments a and b is the series value
# 1 / (1/kappa_a + 1/kappa_b); an infinite entry contributes nothing.
NO_MEMBRANE = math.inf


# --------------------------------------------------------------------------
# Structured Kuhn grid
# --------------------------------------------------------------------------
def kuhn_grid(nx: int, ny: int, nz: int, lo, hi):
    """Nodes and positively oriented tetrahedra of an nx*ny*nz Kuhn grid.

    Node (i, j, k) has index i + (nx+1)*(j + (ny+1)*k) (x fastest).  Each cell
    is split into the six tetrahedra that share its (0,0,0)-(1,1,1) diagonal,
    one per axis permutation, identical in every cell.
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    zs = np.linspace(lo[2], hi[2], nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    sx, sy, sz = 1, nx + 1, (nx + 1) * (ny + 1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = (i * sx + j * sy + k * sz).ravel().astype(np.int64)
    step = np.array([sx, sy, sz], dtype=np.int64)
    perms = [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)]
    tets = []
    for p in perms:
        even = p in [(0, 1, 2), (1, 2, 0), (2, 0, 1)]
        v0 = base
        v1 = v0 + step[p[0]]
        v2 = v1 + step[p[1]]
        v3 = v2 + step[p[2]]
        tets.append(np.stack([v0, v1, v2, v3] if even else [v0, v1, v3, v2], axis=1))
    # cell-major order: the six tetrahedra of a cell are consecutive
    tets = np.stack(tets, axis=1).reshape(-1, 4)
    return xyz, tets.astype(np.int32)


def tet_centroids(xyz, tets):
    return xyz[tets].mean(axis=1)


# --------------------------------------------------------------------------
# Compartment labelling (centroid rule)
# --------------------------------------------------------------------------
def label_sphere(xyz, tets, center, radius):
    c = tet_centroids(xyz, tets)
    inside = ((c - np.asarray(center)) ** 2).sum(axis=1) < radius * radius
    return inside.astype(np.int32)


def place_cylinders_periodic(n: int, L: float, mean_r: float, sigma: float, seed: int,
                             max_trials: int = 100_000):
    """Non-overlapping z-parallel cylinders in a periodic L x L square.

    Radii are lognormal with log-space sd `sigma` and arithmetic mean `mean_r`
    (mu = ln(mean_r) - sigma^2/2).  Cylinders are placed largest first at
    uniform random centres; a centre is accepted when its periodic
    minimum-image distance to every placed centre is at least r_i + r_j.
    If one cylinder cannot be placed in `max_trials` draws the whole packing
    is redrawn with seed + 1.  Returns (centres [n,2], radii [n], seed used).
    """
    s = seed
    while True:
        rng = np.random.default_rng(s)
        mu = math.log(mean_r) - 0.5 * sigma * sigma
        r = np.sort(rng.lognormal(mu, sigma, n))[::-1].copy()
        cen = np.zeros((0, 2))
        ok = True
        for ri in r:
            placed = False
            tried = 0
            while tried < max_trials:
                b = min(4096, max_trials - tried)
                cand = rng.uniform(0.0, L, size=(b, 2))
                tried += b
                if len(cen) == 0:
                    cen = cand[:1]
                    placed = True
                    break
                d = cand[:, None, :] - cen[None, :, :]
                d -= L * np.round(d / L)
                dist = np.sqrt((d ** 2).sum(-1))
                good = np.all(dist >= ri + r[: len(cen)][None, :], axis=1)
                idx = np.flatnonzero(good)
                if idx.size:
                    cen = np.vstack([cen, cand[idx[0]]])
                    placed = True
                    break
            if not placed:
                ok = False
                break
        if ok:
            return cen, r, s
        s += 1


def label_cylinders_periodic(xyz, tets, centres, radii, L):
    c = tet_centroids(xyz, tets)[:, :2]
    lab = np.zeros(len(tets), dtype=np.int32)
    for m, (cc, r) in enumerate(zip(centres, radii)):
        d = c - cc
        d -= L * np.round(d / L)
        inside = (d ** 2).sum(1) < r * r
        lab[inside & (lab == 0)] = m + 1
    return lab


def place_objects(n: int, L: float, rmin: float, rmax: float, gap: float, seed: int,
                  max_trials: int = 10_000):
    """Random non-overlapping spheres and finite cylinders in an L-cube.

    Each object draws its radius r ~ U(rmin, rmax) and its kind (sphere or
    cylinder, 50/50).  A cylinder has length 2r and a random unit axis.  The
    overlap test uses bounding spheres (radius r for a sphere, r*sqrt(2) for a
    cylinder) separated by at least `gap`.  Objects are placed largest first at
    uniform random centres inside the cube; an object that cannot be placed in
    `max_trials` draws is dropped.  Returns a list of dicts.
    """
    rng = np.random.default_rng(seed)
    r = rng.uniform(rmin, rmax, n)
    kind = rng.integers(0, 2, n)  # 0 sphere, 1 cylinder
    ax = rng.normal(size=(n, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    rb = np.where(kind == 1, r * math.sqrt(2.0), r)
    order = np.argsort(-rb, kind="stable")
    placed = []
    cen = np.zeros((0, 3))
    rbp = np.zeros(0)
    for o in order:
        tried = 0
        while tried < max_trials:
            b = min(2048, max_trials - tried)
            cand = rng.uniform(0.0, L, size=(b, 3))
            tried += b
            if len(cen):
                dist = np.sqrt(((cand[:, None, :] - cen[None]) ** 2).sum(-1))
                good = np.all(dist >= rb[o] + rbp[None, :] + gap, axis=1)
                idx = np.flatnonzero(good)
            else:
                idx = np.array([0])
            if idx.size:
                c = cand[idx[0]]
                cen = np.vstack([cen, c])
                rbp = np.append(rbp, rb[o])
                placed.append({"kind": int(kind[o]), "r": float(r[o]), "c": c.copy(),
                               "axis": ax[o].copy()})
                break
    return placed


def label_objects(xyz, tets, objects, h: float, n_cells: int, lo):
    """Centroid rule: a tetrahedron belongs to object m+1 when its centroid is
    inside object m (spheres: |x-c| < r; cylinders: radial distance < r and
    |axial| < r).  Objects do not overlap, so the label is unique."""
    c = tet_centroids(xyz, tets)
    lab = np.zeros(len(tets), dtype=np.int32)
    lo = np.asarray(lo, dtype=np.float64)
    # tetrahedra are cell-major (6 per cell), cells x-fastest
    for m, ob in enumerate(objects):
        rb = ob["r"] * (math.sqrt(2.0) if ob["kind"] == 1 else 1.0)
        i0 = np.clip(np.floor((ob["c"] - rb - lo) / h).astype(int), 0, n_cells - 1)
        i1 = np.clip(np.floor((ob["c"] + rb - lo) / h).astype(int), 0, n_cells - 1)
        kk, jj, ii = np.meshgrid(np.arange(i0[2], i1[2] + 1), np.arange(i0[1], i1[1] + 1),
                                 np.arange(i0[0], i1[0] + 1), indexing="ij")
        cells = (ii + n_cells * (jj + n_cells * kk)).ravel()
        t = (cells[:, None] * 6 + np.arange(6)[None, :]).ravel()
        d = c[t] - ob["c"]
        if ob["kind"] == 0:
            inside = (d ** 2).sum(1) < ob["r"] ** 2
        else:
            a = d @ ob["axis"]
            rad2 = (d ** 2).sum(1) - a * a
            inside = (rad2 < ob["r"] ** 2) & (np.abs(a) < ob["r"])
        sel = t[inside & (lab[t] == 0)]
        lab[sel] = m + 1
    return lab


# --------------------------------------------------------------------------
# Gradient directions and sequences
# --------------------------------------------------------------------------
def fibonacci_dirs(n: int):
    """Golden-angle spiral on the unit sphere: z_i = 1 - (2i+1)/n."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    d = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


@dataclass
class Problem:
    """One geometry with its sequence, directions and b-values.

    RHS r = d * n_b + j uses direction dirs[d] and b-value bvals[j]."""
    name: str
    xyz: np.ndarray            # [n_nodes, 3] float64, um
    tets: np.ndarray           # [n_tets, 4] int32, positive orientation ([n, 3] triangles, [n, 2] segments)
    tet_cmpt: np.ndarray       # [n_tets] int32 in [0, n_cmpt)
    D_cmpt: np.ndarray         # [n_cmpt] float64, um^2/us (= mm^2/s)
    kappa_cmpt: np.ndarray     # [n_cmpt] float64, um/us (= m/s); inf = no membrane
    periodic_mask: int         # bit k: axis k periodic
    box_lo: np.ndarray
    box_hi: np.ndarray
    dt: float                  # us
    delta: float               # us
    Delta: float               # us
    TE: float                  # us
    dirs: np.ndarray           # [n_dir, 3] unit vectors
    bvals: np.ndarray          # [n_b] s/mm^2 (= us/um^2)
    theta: float = 0.5
    transformed: bool = False  # True: gauge-transformed frame (needed when periodic)
    meta: dict = field(default_factory=dict)
    # temporal profile other than PGSE: {"kind": "cos_ogse" | "sin_ogse" | "double_pgse" |
    # "trapezoid" | "double_trapezoid", "n_periods": int, "ramp": us}; None = PGSE
    profile: dict | None = None
    # transverse relaxation 1/T2 (1/us) and initial magnetization per compartment; None = 0 / 1
    inv_T2: np.ndarray | None = None
    rho: np.ndarray | None = None
    # anisotropic diffusion: [n_cmpt, 6] (xx, yy, zz, xy, yz, zx) in mm^2/s; None = isotropic D_cmpt
    D_tensor: np.ndarray | None = None
    # cell-based tensors: [n_tets, 6], one per element (overrides D_tensor); None = per compartment
    D_tensor_elem: np.ndarray | None = None
    # weak pseudo-periodic conditions on a non-periodic box (lab frame):
    # {"axes": bit mask, "kappa_e": um/us or None for max D / h}
    weak_periodic: dict | None = None
    # triangles of a thin layer embedded in 3-D (a 2-D manifold) instead of a planar 2-D domain
    surface: bool = False

    @property
    def n_cmpt(self):
        return len(self.D_cmpt)

    @property
    def n_rhs(self):
        return len(self.dirs) * len(self.bvals)

    @property
    def n_steps(self):
        return int(round(self.TE / self.dt))


def cfg1(n: int = 24, dt: float = 50.0):
    L = 40.0
    lo, hi = np.full(3, -L / 2), np.full(3, L / 2)
    xyz, tets = kuhn_grid(n, n, n, lo, hi)
    return Problem("cfg1", xyz, tets, np.zeros(len(tets), np.int32), np.array([2e-3]),
                   np.array([NO_MEMBRANE]), 0, lo, hi, dt, 2500.0, 5000.0, 7500.0,
                   np.array([[1.0, 0.0, 0.0]]), np.array([1000.0]))


def cfg2(n: int = 48, dt: float = 50.0, bvals=(0.0, 500.0, 1000.0, 2000.0, 3000.0),
         kappa: float = 1e-5):
    L = 20.0
    lo, hi = np.full(3, -L / 2), np.full(3, L / 2)
    xyz, tets = kuhn_grid(n, n, n, lo, hi)
    lab = label_sphere(xyz, tets, np.zeros(3), 5.0)
    return Problem("cfg2", xyz, tets, lab, np.array([2e-3, 2e-3]),
                   np.array([NO_MEMBRANE, kappa]), 0, lo, hi, dt, 2500.0, 5000.0, 7500.0,
                   np.array([[1.0, 0.0, 0.0]]), np.asarray(bvals, dtype=np.float64))


def cfg3(n: int = 64, dt: float = 50.0, n_dir: int = 64, n_b: int = 8, seed: int = 0):
    L = 30.0
    lo, hi = np.zeros(3), np.full(3, L)
    cen, rad, used = place_cylinders_periodic(40, L, 2.0, 0.3, seed)
    xyz, tets = kuhn_grid(n, n, n, lo, hi)
    lab = label_cylinders_periodic(xyz, tets, cen, rad, L)
    nc = len(rad) + 1
    D = np.full(nc, 2e-3)
    kap = np.full(nc, 5e-5)
    kap[0] = NO_MEMBRANE
    return Problem("cfg3", xyz, tets, lab, D, kap, 7, lo, hi, dt, 2500.0, 5000.0, 7500.0,
                   fibonacci_dirs(n_dir), np.linspace(0.0, 3000.0, n_b), transformed=True,
                   meta={"cyl_centres": cen, "cyl_radii": rad, "seed_used": used})


def cfg4(n: int = 96, dt: float = 50.0, n_dir: int = 32, bvals=(500.0, 1000.0, 2000.0, 3000.0),
         seed: int = 0, n_obj: int = 200):
    L = 40.0
    lo, hi = np.zeros(3), np.full(3, L)
    h_ref = L / 96.0
    objs = place_objects(n_obj, L, 1.0, 4.0, h_ref, seed)
    xyz, tets = kuhn_grid(n, n, n, lo, hi)
    lab = label_objects(xyz, tets, objs, L / n, n, lo)
    rng = np.random.default_rng(seed + 1)
    nc = len(objs) + 1
    kap = np.concatenate([[NO_MEMBRANE], rng.uniform(1e-5, 1e-4, nc - 1)])
    D = np.full(nc, 2e-3)
    return Problem("cfg4", xyz, tets, lab, D, kap, 0, lo, hi, dt, 2500.0, 5000.0, 7500.0,
                   fibonacci_dirs(n_dir), np.asarray(bvals, dtype=np.float64),
                   meta={"objects": objs, "n_placed": len(objs)})


def cfg5_geometry(g: int, dt: float = 50.0, n_dir: int = 16,
                  bvals=(500.0, 1000.0, 2000.0, 3000.0), scale: float = 1.0):
    """Geometry g (0..31) of the uneven batch.  Node count n ~ log-uniform
    [50k, 2M]; grid N = round(n^(1/3)) - 1 (times `scale` for reduced copies);
    box side N * 40/96 um (the cfg4 cell size); objects as in cfg4 with a count
    proportional to the box volume; PGSE delta ~ U(2, 10) ms,
    Delta ~ U(max(delta, 5), 40) ms, both rounded to dt."""
    rng = np.random.default_rng(5000 + g)
    nn = math.exp(rng.uniform(math.log(5e4), math.log(2e6)))
    N = int(round(nn ** (1.0 / 3.0))) - 1
    L = N * 40.0 / 96.0
    n_obj = max(1, int(round(200 * (L / 40.0) ** 3)))
    objs = place_objects(n_obj, L, 1.0, 4.0, 40.0 / 96.0, 5000 + g)
    delta = rng.uniform(2000.0, 10000.0)
    Delta = rng.uniform(max(delta, 5000.0), 40000.0)
    delta = max(dt, round(delta / dt) * dt)
    Delta = max(delta, round(Delta / dt) * dt)
    Ng = max(2, int(round(N * scale)))
    lo, hi = np.zeros(3), np.full(3, L)
    xyz, tets = kuhn_grid(Ng, Ng, Ng, lo, hi)
    lab = label_objects(xyz, tets, objs, L / Ng, Ng, lo)
    nc = len(objs) + 1
    kap = np.concatenate([[NO_MEMBRANE], rng.uniform(1e-5, 1e-4, nc - 1)])
    D = np.full(nc, 2e-3)
    return Problem(f"cfg5_g{g}", xyz, tets, lab, D, kap, 0, lo, hi, dt, delta, Delta,
                   Delta + delta, fibonacci_dirs(n_dir), np.asarray(bvals, dtype=np.float64),
                   meta={"N": N, "n_placed": len(objs)})


def free_periodic_box(n: int = 8, L: float = 10.0, dt: float = 50.0, D: float = 2e-3,
                      dirs=((1.0, 0.0, 0.0),), bvals=(1000.0,)):
    """Periodic box without compartments (free diffusion)."""
    lo, hi = np.zeros(3), np.full(3, L)
    xyz, tets = kuhn_grid(n, n, n, lo, hi)
    return Problem("free_periodic", xyz, tets, np.zeros(len(tets), np.int32), np.array([D]),
                   np.array([NO_MEMBRANE]), 7, lo, hi, dt, 2500.0, 5000.0, 7500.0,
                   np.asarray(dirs, dtype=np.float64), np.asarray(bvals, dtype=np.float64),
                   transformed=True)


def slab_1d(nx: int, L: float = 40.0, w: float = 1.0, dt: float = 50.0, D: float = 2e-3,
            b: float = 1000.0, delta: float = 2500.0, Delta: float = 5000.0):
    """[-L/2, L/2] x [0, w] x [0, w] Neumann box with nx x 1 x 1 Kuhn cells and
    the gradient along x: the continuum signal equals that of the 1-D interval."""
    lo = np.array([-L / 2, 0.0, 0.0])
    hi = np.array([L / 2, w, w])
    xyz, tets = kuhn_grid(nx, 1, 1, lo, hi)
    return Problem("slab1d", xyz, tets, np.zeros(len(tets), np.int32), np.array([D]),
                   np.array([NO_MEMBRANE]), 0, lo, hi, dt, delta, Delta, Delta + delta,
                   np.array([[1.0, 0.0, 0.0]]), np.array([b]))


def kuhn_grid_2d(nx: int, ny: int, lo, hi):
    """Nodes (z = 0) and counter-clockwise triangles of an nx*ny grid of the
    rectangle [lo, hi] (x, y): each cell is split along its (0,0)-(1,1)
    diagonal, identically in every cell.  Node (i, j) has index i + (nx+1) j."""
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    v00 = (i + (nx + 1) * j).ravel()
    v10, v01 = v00 + 1, v00 + nx + 1
    v11 = v01 + 1
    tris = np.stack([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], axis=1).reshape(-1, 3)
    return xyz, tris.astype(np.int32)


def square_disk(n: int = 40, L: float = 10.0, R: float = 3.0, dt: float = 50.0, kappa: float = 1e-5,
                bvals=(0.0, 1000.0, 3000.0), dirs=((1.0, 0.0, 0.0),)):
    """2-D: a disk of radius R (compartment 1, centroid rule, permeable membrane)
    centred in the square [-L/2, L/2]^2 (compartment 0), Neumann outer
    boundary; the paper's two-dimensional disk experiments at reduced size."""
    lo2, hi2 = np.full(2, -L / 2), np.full(2, L / 2)
    xyz, tris = kuhn_grid_2d(n, n, lo2, hi2)
    cen = xyz[tris].mean(axis=1)
    lab = (np.hypot(cen[:, 0], cen[:, 1]) < R).astype(np.int32)
    lo, hi = np.array([lo2[0], lo2[1], -1.0]), np.array([hi2[0], hi2[1], 1.0])
    return Problem("square_disk", xyz, tris, lab, np.array([2e-3, 2e-3]), np.array([NO_MEMBRANE, kappa]), 0,
                   lo, hi, dt, 2500.0, 5000.0, 7500.0, np.asarray(dirs, dtype=np.float64),
                   np.asarray(bvals, dtype=np.float64))


def polar_disk(m: int, R: float = 5.0, dt: float = 50.0, D: float = 2e-3, bvals=(1000.0,),
               dirs=((1.0, 0.0, 0.0),), delta: float = 2500.0, Delta: float = 5000.0):
    """2-D: the disk of radius R meshed in m rings (ring i holds 6 i nodes on
    the circle of radius R i / m, plus the centre), neighbouring rings joined
    by walking both in angle; the boundary nodes lie on the circle, so the
    polygon approaches the disk at second order.  One compartment, Neumann."""
    xyz = [np.zeros(3)]
    rings = [[0]]
    for i in range(1, m + 1):
        ang = 2.0 * np.pi * np.arange(6 * i) / (6 * i)
        ids = list(range(len(xyz), len(xyz) + 6 * i))
        xyz += [np.array([R * i / m * math.cos(a), R * i / m * math.sin(a), 0.0]) for a in ang]
        rings.append(ids)
    xyz = np.array(xyz)
    tris = []
    for i in range(1, m + 1):
        inner, outer = rings[i - 1], rings[i]
        if i == 1:
            tris += [(0, outer[j], outer[(j + 1) % 6]) for j in range(6)]
            continue
        ni, no = len(inner), len(outer)
        a = b = 0
        while a < ni or b < no:
            ta = 2.0 * np.pi * (a + 1) / ni            # angle of the next inner node
            tb = 2.0 * np.pi * (b + 1) / no            # angle of the next outer node
            if b < no and (a >= ni or tb <= ta):
                tris.append((inner[a % ni], outer[b % no], outer[(b + 1) % no]))
                b += 1
            else:
                tris.append((inner[a % ni], outer[b % no], inner[(a + 1) % ni]))
                a += 1
    tris = np.array(tris, dtype=np.int32)
    X = xyz[tris]
    area2 = (X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1]) - (X[:, 1, 1] - X[:, 0, 1]) * (X[:, 2, 0] - X[:, 0, 0])
    tris[area2 < 0] = tris[area2 < 0][:, [0, 2, 1]]            # counter-clockwise
    lo, hi = np.array([-R, -R, -1.0]), np.array([R, R, 1.0])
    return Problem("polar_disk", xyz, tris, np.zeros(len(tris), np.int32), np.array([D]), np.array([NO_MEMBRANE]),
                   0, lo, hi, dt, delta, Delta, Delta + delta, np.asarray(dirs, dtype=np.float64),
                   np.asarray(bvals, dtype=np.float64))


def periodic_cylinder(m: int, nz: int = 2, R: float = 5.0, H: float = 2.0, dt: float = 50.0, D: float = 2e-3,
                      bvals=(1000.0,), dirs=((1.0, 0.0, 0.0),)):
    """3-D: the polar disk of `polar_disk` extruded into nz layers over a height
    H that is periodic in z (transformed frame), each prism cut into three
    tetrahedra by the order of its triangle's global vertex ids (so shared
    quadrilateral faces are cut the same way from both sides).  For gradients
    across the axis the signal is the disk's."""
    d = polar_disk(m, R=R)
    nn = len(d.xyz)
    z = np.linspace(0.0, H, nz + 1)
    xyz = np.concatenate([np.column_stack([d.xyz[:, :2], np.full(nn, zk)]) for zk in z])
    tets = []
    for tri in np.sort(d.tets, axis=1):
        a, b, c = tri
        for k in range(nz):
            lo, up = k * nn, (k + 1) * nn
            tets += [(a + lo, b + lo, c + lo, a + up), (b + lo, c + lo, a + up, b + up),
                     (c + lo, a + up, b + up, c + up)]
    tets = np.array(tets, dtype=np.int32)
    X = xyz[tets]
    vol = np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))
    tets[vol < 0] = tets[vol < 0][:, [0, 1, 3, 2]]
    lo, hi = np.array([-R, -R, 0.0]), np.array([R, R, H])
    return Problem("periodic_cylinder", xyz, tets, np.zeros(len(tets), np.int32), np.array([D]),
                   np.array([NO_MEMBRANE]), 4, lo, hi, dt, 2500.0, 5000.0, 7500.0,
                   np.asarray(dirs, dtype=np.float64), np.asarray(bvals, dtype=np.float64), transformed=True)


def layered_disk(n: int = 40, radii=(5.0, 7.5, 10.0), dt: float = 100.0, D: float = 3e-3, kappa: float = 1e-5,
                 rho=(0.0, 1.0, 0.0), bvals=(0.0, 1000.0, 4000.0), dirs=((1.0, 0.0, 0.0),)):
    """2-D: concentric layers r < radii[0], ..., r < radii[-1] (one compartment
    each, permeable membranes between them, Neumann outside) cut from an n x n
    grid of the square [-R, R]^2, R = radii[-1]: triangles whose centroid lies
    outside R are dropped and the unused nodes removed.  The paper's
    three-layer disk with the initial magnetization rho per layer, its PGSE
    (delta 10.6 ms, Delta 43.1 ms) on a 100 us grid."""
    R = radii[-1]
    xyz, tris = kuhn_grid_2d(n, n, np.full(2, -R), np.full(2, R))
    r = np.hypot(*xyz[tris].mean(axis=1)[:, :2].T)
    tris = tris[r < R]
    r = r[r < R]
    used = np.unique(tris)
    new_id = np.full(len(xyz), -1, np.int64)
    new_id[used] = np.arange(len(used))
    xyz, tris = xyz[used], new_id[tris].astype(np.int32)
    lab = np.searchsorted(np.asarray(radii[:-1], float), r, side="right").astype(np.int32)
    nc = len(radii)
    lo, hi = np.array([-R, -R, -1.0]), np.array([R, R, 1.0])
    p = Problem("layered_disk", xyz, tris, lab, np.full(nc, D), np.full(nc, kappa), 0, lo, hi, dt, 10600.0,
                43100.0, 53700.0, np.asarray(dirs, dtype=np.float64), np.asarray(bvals, dtype=np.float64))
    p.rho = np.asarray(rho, dtype=np.float64)
    return p


def _keep_elements(xyz, tets, keep):
    """The elements `keep` and the nodes they use, renumbered."""
    tets = tets[keep]
    used = np.unique(tets)
    new_id = np.full(len(xyz), -1, np.int64)
    new_id[used] = np.arange(len(used))
    return xyz[used], new_id[tets].astype(np.int32)


def layered_sphere(n: int = 16, radii=(5.0, 7.5, 10.0), dt: float = 100.0, D=(3e-3, 1e-3, 3e-3),
                   kappa: float = 1e-5, bvals=(1000.0, 4000.0), dirs=((1.0, 0.0, 0.0),)):
    """3-D: concentric shells r < radii[0] < ... < radii[-1] (one compartment
    each, permeable membranes, Neumann outside) cut from an n^3 Kuhn grid of
    the cube [-R, R]^3 by tetrahedron centroids; the paper's three-layer
    sphere with its per-layer diffusivities and neuron PGSE (100 us grid)."""
    R = radii[-1]
    xyz, tets = kuhn_grid(n, n, n, np.full(3, -R), np.full(3, R))
    r = np.linalg.norm(xyz[tets].mean(axis=1), axis=1)
    xyz, tets = _keep_elements(xyz, tets, r < R)
    r = np.linalg.norm(xyz[tets].mean(axis=1), axis=1)
    lab = np.searchsorted(np.asarray(radii[:-1], float), r, side="right").astype(np.int32)
    nc = len(radii)
    return Problem("layered_sphere", xyz, tets, lab, np.asarray(D, float), np.full(nc, kappa), 0, np.full(3, -R),
                   np.full(3, R), dt, 10600.0, 43100.0, 53700.0, np.asarray(dirs, dtype=np.float64),
                   np.asarray(bvals, dtype=np.float64))


def layered_torus(h: float = 2.0, R_ring: float = 20.0, radii=(5.0, 7.5, 10.0), dt: float = 100.0,
                  D=(3e-3, 1e-3, 3e-3), kappa: float = 1e-5, bvals=(1000.0, 4000.0), dirs=((1.0, 0.0, 0.0),)):
    """3-D: a torus whose tube (distance rho to the circle of radius R_ring in
    the xy plane) is layered rho < radii[0] < ... < radii[-1], cut from a
    Kuhn grid of spacing about h; the paper's three-layer torus."""
    a = radii[-1]
    lo = np.array([-(R_ring + a), -(R_ring + a), -a])
    hi = -lo
    nx = int(round((hi[0] - lo[0]) / h))
    nz = int(round((hi[2] - lo[2]) / h))
    xyz, tets = kuhn_grid(nx, nx, nz, lo, hi)

    def tube_dist(c):
        return np.hypot(np.hypot(c[:, 0], c[:, 1]) - R_ring, c[:, 2])
    rho = tube_dist(xyz[tets].mean(axis=1))
    xyz, tets = _keep_elements(xyz, tets, rho < a)
    rho = tube_dist(xyz[tets].mean(axis=1))
    lab = np.searchsorted(np.asarray(radii[:-1], float), rho, side="right").astype(np.int32)
    nc = len(radii)
    return Problem("layered_torus", xyz, tets, lab, np.asarray(D, float), np.full(nc, kappa), 0, lo, hi, dt,
                   10600.0, 43100.0, 53700.0, np.asarray(dirs, dtype=np.float64), np.asarray(bvals, dtype=np.float64))


def free_periodic_square(n: int = 8, L: float = 10.0, dt: float = 50.0, D: float = 2e-3,
                         dirs=((1.0, 0.0, 0.0),), bvals=(1000.0,)):
    """2-D periodic square without compartments (free diffusion)."""
    xyz, tris = kuhn_grid_2d(n, n, np.zeros(2), np.full(2, L))
    lo, hi = np.array([0.0, 0.0, -1.0]), np.array([L, L, 1.0])
    return Problem("free_periodic_square", xyz, tris, np.zeros(len(tris), np.int32), np.array([D]),
                   np.array([NO_MEMBRANE]), 3, lo, hi, dt, 2500.0, 5000.0, 7500.0,
                   np.asarray(dirs, dtype=np.float64), np.asarray(bvals, dtype=np.float64), transformed=True)


def sheared_box(n: int = 6, L: float = 8.0, eps: float = 0.3, dt: float = 50.0, D: float = 2e-3,
                dirs=((1.0, 0.0, 0.0),), bvals=(1000.0,)):
    """A free box [0, L]^3 meshed without periodicity whose x sides do not
    match: every node moves along y by eps sin(pi y / L) x / L, so nodes stay
    on their box planes, the x = 0 side is untouched and the x = L side's
    nodes slide along y (a shear smaller than half a cell keeps every
    tetrahedron positive)."""
    p = free_periodic_box(n=n, L=L, dt=dt, D=D, dirs=dirs, bvals=bvals)
    x, y = p.xyz[:, 0], p.xyz[:, 1]
    p.xyz = p.xyz.copy()
    p.xyz[:, 1] = y + eps * np.sin(np.pi * y / L) * x / L
    p.periodic_mask = 0
    p.transformed = False
    p.name = "sheared_box"
    return p


def line_segments(n: int, L: float = 40.0, direction=(1.0, 0.0, 0.0), dt: float = 50.0, D: float = 2e-3,
                  bvals=(1000.0,), dirs=((1.0, 0.0, 0.0),), delta: float = 2500.0, Delta: float = 5000.0):
    """1-D manifold: a straight fibre of length L along `direction`, centred at
    the origin, cut into n equal P1 segments (Neumann ends)."""
    t = np.asarray(direction, float)
    t = t / np.linalg.norm(t)
    s = np.linspace(-L / 2, L / 2, n + 1)
    xyz = s[:, None] * t[None, :]
    segs = np.stack([np.arange(n), np.arange(1, n + 1)], axis=1).astype(np.int32)
    lo, hi = np.full(3, -L / 2), np.full(3, L / 2)
    return Problem("line", xyz, segs, np.zeros(n, np.int32), np.array([D]), np.array([NO_MEMBRANE]), 0, lo, hi,
                   dt, delta, Delta, Delta + delta, np.asarray(dirs, dtype=np.float64),
                   np.asarray(bvals, dtype=np.float64))


def dendrite_tree(seed: int = 0, n_stems: int = 6, depth: int = 5, h: float = 1.0, length=(15.0, 40.0),
                  dt: float = 100.0, D: float = 2e-3, bvals=(0.0, 1000.0, 3000.0), n_dir: int = 3):
    """1-D manifold standing in for a neuron's dendrite tree: n_stems primary
    branches leave a soma point at the origin in random directions; every
    branch bends slightly along its length and splits into two children
    turned 25-60 degrees away from it, down to `depth` levels.  Branch lengths
    are uniform in `length`, segments about h long; one compartment.  The
    sequence is the paper's neuron PGSE (delta 10.6 ms, Delta 43.1 ms), whose
    TE = 53.7 ms is a multiple of dt = 100 us."""
    rng = np.random.default_rng(seed)
    xyz = [np.zeros(3)]
    segs = []

    def unit(v):
        return v / np.linalg.norm(v)

    def turn(d, lo_deg, hi_deg):
        a = math.radians(rng.uniform(lo_deg, hi_deg))
        w = unit(np.cross(d, rng.normal(size=3)))
        return unit(math.cos(a) * d + math.sin(a) * w)

    stack = [(0, unit(rng.normal(size=3)), 1) for _ in range(n_stems)]
    while stack:
        v0, d, level = stack.pop()
        n = max(2, int(round(rng.uniform(*length) / h)))
        v = v0
        for _ in range(n):
            d = turn(d, 0.0, 8.0)
            xyz.append(xyz[v] + h * d)
            segs.append((v, len(xyz) - 1))
            v = len(xyz) - 1
        if level < depth:
            stack += [(v, turn(d, 25.0, 60.0), level + 1), (v, turn(d, 25.0, 60.0), level + 1)]
    xyz = np.array(xyz)
    segs = np.array(segs, dtype=np.int32)
    lo, hi = xyz.min(axis=0) - h, xyz.max(axis=0) + h
    return Problem("dendrite_tree", xyz, segs, np.zeros(len(segs), np.int32), np.array([D]),
                   np.array([NO_MEMBRANE]), 0, lo, hi, dt, 10600.0, 43100.0, 53700.0, fibonacci_dirs(n_dir),
                   np.asarray(bvals, dtype=np.float64))


def icosphere(level: int, R: float = 1.0):
    """Nodes on the sphere of radius R and triangles of the icosahedron refined
    `level` times (each triangle cut into four, new nodes pushed to the
    sphere), outward-oriented."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    xyz = [np.array(p, float) / np.linalg.norm(p) for p in v]
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = xyz[a] + xyz[b]
                xyz.append(m / np.linalg.norm(m))
                mid[key] = len(xyz) - 1
            return mid[key]
        nf = []
        for a, b, c in f:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    return R * np.array(xyz), np.array(f, dtype=np.int32)


def spherical_shell(level: int = 4, R: float = 5.0, dt: float = 50.0, D: float = 2e-3, kappa: float | None = None,
                    cap_z: float = 0.5, bvals=(0.0, 1000.0, 3000.0), dirs=((1.0, 0.0, 0.0), (0.0, 0.0, 1.0))):
    """Thin layer: the sphere of radius R as a 2-D manifold of triangles.  With
    kappa given, triangles whose centroid has z > cap_z R form a second
    compartment, separated from the rest by a permeable membrane along the
    circle of latitude (a curve on the surface)."""
    xyz, tris = icosphere(level, R)
    lab = np.zeros(len(tris), np.int32)
    D_c, k_c = np.array([D]), np.array([NO_MEMBRANE])
    if kappa is not None:
        lab = (xyz[tris].mean(axis=1)[:, 2] > cap_z * R).astype(np.int32)
        D_c, k_c = np.array([D, D]), np.array([NO_MEMBRANE, kappa])
    lo, hi = np.full(3, -R), np.full(3, R)
    d = np.asarray(dirs, dtype=np.float64)
    return Problem("spherical_shell", xyz, tris, lab, D_c, k_c, 0, lo, hi, dt, 2500.0, 5000.0, 7500.0,
                   d / np.linalg.norm(d, axis=1, keepdims=True), np.asarray(bvals, dtype=np.float64), surface=True)


def union(problems, name="batch"):
    """Disjoint union of several geometries as one input mesh (the uneven
    batch): each geometry is translated so that its box centre sits at the
    origin (the origin of g.x is then each geometry's own centre), node and
    compartment ids are offset, and the PGSE timing of each geometry is kept
    in `segments`.  All geometries must share dt and the directions/b-values
    (the first problem's are used)."""
    xyz, tets, cmpt, D, kap = [], [], [], [], []
    node_off, c_off = [0], 0
    half = 0.0
    for p in problems:
        c = 0.5 * (np.asarray(p.box_lo) + np.asarray(p.box_hi))
        xyz.append(p.xyz - c)
        tets.append(p.tets + node_off[-1])
        cmpt.append(p.tet_cmpt + c_off)
        D.append(p.D_cmpt)
        kap.append(p.kappa_cmpt)
        node_off.append(node_off[-1] + len(p.xyz))
        c_off += p.n_cmpt
        half = max(half, float(np.max(np.asarray(p.box_hi) - c)))
    p0 = problems[0]
    if len({p.tets.shape[1] for p in problems}) != 1 or len({p.surface for p in problems}) != 1:
        raise ValueError("a batch holds one element family")
    out = Problem(name, np.concatenate(xyz), np.concatenate(tets).astype(np.int32),
                  np.concatenate(cmpt).astype(np.int32), np.concatenate(D), np.concatenate(kap), 0,
                  np.full(3, -half), np.full(3, half), p0.dt, p0.delta, p0.Delta, p0.TE, p0.dirs, p0.bvals,
                  surface=p0.surface)
    out.segments = {"node_off": np.array(node_off, dtype=np.int64),
                    "delta": np.array([p.delta for p in problems]),
                    "Delta": np.array([p.Delta for p in problems]),
                    "TE": np.array([p.TE for p in problems])}
    return out


def cfg5(n_geom: int = 32, scale: float = 1.0, dt: float = 50.0):
    """The uneven batch: geometries 0..n_geom-1 of cfg5_geometry (grids scaled
    by `scale` for reduced copies) as one union mesh."""
    return union([cfg5_geometry(g, dt=dt, scale=scale) for g in range(n_geom)], name="cfg5")

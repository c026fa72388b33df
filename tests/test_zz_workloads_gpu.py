"""GPU parity cases over the wider workloads: full-size properties of the
benchmarked cfg4 workload and of the 64-tree forest, every element family
under each Krylov variant, the paper's settings (Section 4), cell-based
tensors and the textbook references (disk, shell, extruded cylinder), each
against the CPU FP64 oracle.  Tolerances as in test_gpu_parity.py: plain FP64
1e-10, mixed 1e-6 (relative)."""
import numpy as np
import pytest

import geom
import oracle
from oracle import btoracle as bo

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def bt():
    from paper_1908_01719_gb300 import build, bt as btmod
    build.build()
    return btmod


@pytest.fixture(scope="module")
def sim_cls(bt):
    from paper_1908_01719_gb300.simulate import Simulation
    return Simulation


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def _tree():
    return geom.dendrite_tree(seed=4, n_stems=4, depth=4, length=(10.0, 25.0))


def _shell():
    return geom.spherical_shell(level=3, R=5.0, kappa=1e-4, cap_z=0.3, bvals=(0.0, 1000.0, 3000.0),
                                dirs=((1.0, 0.0, 0.0), (0.3, -0.5, 0.8)))


# ---------------------------------------------------------------- the benchmarked workload at full size
def test_cfg4_full_size_properties(sim_cls, bt):
    """cfg4 at full size (96^3 Kuhn grid, 1.07 M dofs, 32 directions x 4
    b-values), run as bench.py runs it (mixed mode, autotuned variants,
    captured run graph): sampled RHS against the plain FP64 GPU path (itself
    parity-tested against the oracle above), and, on the same geometry, the
    b = 0 signal equal to the box volume at every direction (conservation,
    exact at any size)."""
    p = geom.cfg4()
    sim = sim_cls(p)
    try:
        S, err, stat, _ = sim.run(bt.BT_MODE_MIXED)
        assert np.all(stat == 0)
        for r in (0, p.n_rhs - 1):
            S64, _, st64, _ = sim.run(bt.BT_MODE_PLAIN_FP64, rhs_begin=r, rhs_end=r + 1)
            assert st64[r] == 0
            assert rel(S[r], S64[r]) < TOL_MIXED, (r, S[r], S64[r])
    finally:
        sim.close()
    import dataclasses
    q = dataclasses.replace(p, dirs=p.dirs[:2].copy(), bvals=np.array([0.0, 3000.0]))
    sim = sim_cls(q)
    try:
        S, err, stat, _ = sim.run(bt.BT_MODE_MIXED)
        assert np.all(stat == 0)
        vol = float(np.prod(np.asarray(q.box_hi) - np.asarray(q.box_lo)))
        assert np.max(np.abs(S[::2] - vol)) < 1e-9 * vol, S[::2]
        assert np.all(np.abs(S[1::2]) < vol)
    finally:
        sim.close()


def test_dendrite_forest_full_size_sampled_against_oracle(sim_cls, bt):
    """The 1-D workload at full size (64 seeded dendrite trees as one uneven
    batch, 537 steps, 9 RHS each), mixed mode as benchmarked: sampled trees
    against the oracle, and every tree's b = 0 signals equal its length
    (conservation, any size)."""
    trees = [geom.dendrite_tree(seed=s) for s in range(64)]
    u = geom.union(trees, name="trees1d")
    sim = sim_cls(u)
    try:
        S, err, stat, _ = sim.run(bt.BT_MODE_MIXED)
    finally:
        sim.close()
    assert np.all(stat == 0)
    R = trees[0].n_rhs
    for g in (0, 21, 42, 63):
        ref = oracle.run(trees[g])
        assert np.max(np.abs(S[g * R:(g + 1) * R] - ref) / np.abs(ref)) < 1e-6, g
    nb = len(trees[0].bvals)
    for g, t in enumerate(trees):
        length = np.linalg.norm(t.xyz[t.tets[:, 1]] - t.xyz[t.tets[:, 0]], axis=1).sum()
        s0 = S[g * R:(g + 1) * R][::nb]                    # b = 0 of each direction
        assert np.max(np.abs(s0 - length)) < 1e-6 * length, g


# ---------------------------------------------------------------- every element family under each variant
FAMILIES = {
    "disk2d": lambda: geom.square_disk(n=16, L=10.0, R=3.0, kappa=1e-4, bvals=(0.0, 1000.0, 3000.0),
                                       dirs=((1.0, 0.0, 0.0), (0.6, 0.8, 0.0))),
    "tree": lambda: _tree(),
    "shell": lambda: _shell(),
}


@pytest.fixture(scope="module")
def family_field():
    cache = {}

    def get(name):
        if name not in cache:
            p = FAMILIES[name]()
            cache[name] = (p,) + oracle.run(p, return_field=True)
        return cache[name]
    return get


@pytest.mark.parametrize("name", list(FAMILIES))
@pytest.mark.parametrize("variant", ["row", "halo"])
@pytest.mark.parametrize("loop", ["graph", "host"])
def test_element_families_under_each_variant(sim_cls, bt, family_field, name, variant, loop):
    """Planar triangles, manifold segments and surface triangles through both
    inner-Krylov variants and both drivers: signals and every dof of the
    field at TE against the oracle, mixed mode."""
    p, ref, U = family_field(name)
    flags = {"row": bt.BT_OPT_VARIANT_ROW, "halo": bt.BT_OPT_VARIANT_HALO}[variant]
    if loop == "host":
        flags |= bt.BT_OPT_NO_GRAPH
    sim = sim_cls(p)
    try:
        S, err, stat, st = sim.run(bt.BT_MODE_MIXED, flags=flags)
        assert np.all(stat == 0)
        assert rel(S, ref).max() < TOL_MIXED, rel(S, ref)
        for r in range(p.n_rhs):
            u = bt.bt_get_state(sim.ctx, r)
            assert (np.abs(u - U[r]) / np.abs(U[r]).max()).max() < TOL_MIXED, r
    finally:
        sim.close()


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_layered_disk_discontinuous_initial_condition(sim_cls, bt, mode):
    """The paper's three-layer disk with initial magnetization [0, 1, 0], its
    D, kappa and neuron PGSE, against the oracle."""
    p = geom.layered_disk(n=24, bvals=(0.0, 1000.0, 4000.0), dirs=((1.0, 0.0, 0.0), (0.6, 0.8, 0.0)))
    ref = oracle.run(p)
    sim = sim_cls(p)
    try:
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S, err, stat, st = sim.run(m)
        assert np.all(stat == 0)
        tol = TOL_FP64 if mode == "plain" else TOL_MIXED
        assert rel(S, ref).max() < tol, rel(S, ref)
    finally:
        sim.close()


# ---------------------------------------------------------------- cell-based diffusion tensors
def _cell_tensor_cases():
    rng = np.random.default_rng(11)
    p = geom.cfg2(n=8, kappa=1e-4, bvals=(1000.0, 3000.0))
    p.dirs = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]])
    A = rng.normal(size=(len(p.tets), 3, 3)) * 3e-2
    S = np.einsum("nij,nkj->nik", A, A) + 2e-4 * np.eye(3)[None]
    p.D_tensor_elem = np.stack([S[:, 0, 0], S[:, 1, 1], S[:, 2, 2], S[:, 0, 1], S[:, 1, 2], S[:, 2, 0]], axis=1)
    # a 2-D disk whose outer layer diffuses mainly along circles about the centre (tensor from the cell midpoint)
    q = geom.layered_disk(n=24, rho=(1.0, 1.0, 1.0), bvals=(1000.0, 4000.0), dirs=((1.0, 0.0, 0.0),))
    c = q.xyz[q.tets].mean(axis=1)
    rh = c[:, :2] / np.maximum(np.linalg.norm(c[:, :2], axis=1, keepdims=True), 1e-12)
    Dr, Dt = np.where(q.tet_cmpt == 2, 0.3e-3, 3e-3), np.full(len(q.tets), 3e-3)
    xx = Dr * rh[:, 0] ** 2 + Dt * rh[:, 1] ** 2
    yy = Dr * rh[:, 1] ** 2 + Dt * rh[:, 0] ** 2
    xy = (Dr - Dt) * rh[:, 0] * rh[:, 1]
    q.D_tensor_elem = np.stack([xx, yy, Dt, xy, 0 * xx, 0 * xx], axis=1)
    return {"random_spd": p, "radial_disk": q}


@pytest.mark.parametrize("case", ["random_spd", "radial_disk"])
@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_element_tensors_match_oracle(sim_cls, bt, case, mode):
    """One diffusion tensor per element (bt_set_element_tensors): the stiffness
    plane and the signals against the oracle."""
    p = _cell_tensor_cases()[case]
    a = bo.assemble(p)
    ref = oracle.run(p, asm=a)
    sim = sim_cls(p)
    try:
        rp, col = bt.bt_get_pattern(sim.ctx)
        v = bt.bt_get_plane(sim.ctx, "K")
        K = a["K"].tocsr()
        dense = np.zeros_like(v)
        for i in range(len(rp) - 1):
            m = dict(zip(K.getrow(i).indices, K.getrow(i).data))
            dense[rp[i]:rp[i + 1]] = [m.get(c, 0.0) for c in col[rp[i]:rp[i + 1]]]
        assert np.abs(v - dense).max() <= 1e-13 * np.abs(dense).max()
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S, err, stat, st = sim.run(m)
        assert np.all(stat == 0)
        tol = TOL_FP64 if mode == "plain" else TOL_MIXED
        assert rel(S, ref).max() < tol, rel(S, ref)
    finally:
        sim.close()


def test_polar_disk_against_oracle_and_matrix_formalism(sim_cls, bt):
    """A disk meshed with its boundary on the circle: mixed-mode signals against
    the oracle, and within the discretisation error (measured on the CPU) of the
    disk's matrix-formalism value."""
    from oracle import mfdisk
    p = geom.polar_disk(32, dt=12.5)
    ref = oracle.run(p)
    X = p.xyz[p.tets]
    area = 0.5 * np.abs(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])[:, 2]).sum()
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    mf = mfdisk.mf_disk_signal(5.0, 2e-3, q, 2500.0, 5000.0).real
    sim = sim_cls(p)
    try:
        S, err, stat, st = sim.run(bt.BT_MODE_MIXED)
        assert np.all(stat == 0)
        assert rel(S, ref).max() < TOL_MIXED
        assert abs(S[0].real / area - mf) < 2e-5
    finally:
        sim.close()


def test_icosphere_against_oracle_and_matrix_formalism(sim_cls, bt):
    """A thin spherical layer (level-4 icosphere): mixed-mode signals against
    the oracle, and within the discretisation error (measured on the CPU) of
    the shell's matrix-formalism value."""
    from oracle import mfshell
    p = geom.spherical_shell(level=4, R=5.0, dt=12.5, bvals=(1000.0,), dirs=((0.0, 0.0, 1.0),))
    ref = oracle.run(p)
    X = p.xyz[p.tets]
    area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1).sum()
    q = float(oracle.q_from_b(1000.0, 2500.0, 5000.0))
    mf = mfshell.mf_shell_signal(5.0, 2e-3, q, 2500.0, 5000.0).real
    sim = sim_cls(p)
    try:
        S, err, stat, st = sim.run(bt.BT_MODE_MIXED)
        assert np.all(stat == 0)
        assert rel(S, ref).max() < TOL_MIXED
        assert abs(S[0].real / area - mf) < 2e-4
    finally:
        sim.close()


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_periodic_cylinder_against_oracle(sim_cls, bt, mode):
    """Tetrahedra of a disk extruded along a periodic z axis (transformed frame,
    curved Neumann wall): signals against the oracle."""
    p = geom.periodic_cylinder(12, dt=25.0, dirs=((0.6, 0.8, 0.0), (0.0, 0.0, 1.0)), bvals=(1000.0, 3000.0))
    ref = oracle.run(p)
    sim = sim_cls(p)
    try:
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S, err, stat, st = sim.run(m)
        assert np.all(stat == 0)
        tol = TOL_FP64 if mode == "plain" else TOL_MIXED
        assert rel(S, ref).max() < tol, rel(S, ref)
    finally:
        sim.close()


@pytest.mark.parametrize("kind", ["pgse", "double_pgse", "cos_ogse", "sin_ogse", "trapezoid", "double_trapezoid"])
def test_six_profiles_in_a_disk(sim_cls, bt, kind):
    """Section 4's six temporal profiles in a disk of radius 5 um with
    delta = Delta = 10 ms, mixed mode, against the oracle."""
    TE = {"pgse": 20000.0, "double_pgse": 40000.0, "cos_ogse": 20000.0, "sin_ogse": 20000.0,
          "trapezoid": 20000.0, "double_trapezoid": 40000.0}
    p = geom.polar_disk(12, dt=100.0, bvals=(1000.0, 3000.0), dirs=((1.0, 0.0, 0.0), (0.6, 0.8, 0.0)))
    p.delta, p.Delta, p.TE = 10000.0, 10000.0, TE[kind]
    p.profile = {"kind": kind, "n_periods": 1, "ramp": 1000.0}
    ref = oracle.run(p)
    sim = sim_cls(p)
    try:
        S, err, stat, st = sim.run(bt.BT_MODE_MIXED)
        assert np.all(stat == 0)
        assert rel(S, ref).max() < TOL_MIXED, rel(S, ref)
    finally:
        sim.close()


@pytest.mark.parametrize("t2", ["none", "inner", "outer"])
def test_three_layer_t2_cross_section(sim_cls, bt, t2):
    """Section 4's T2 study of a three-layer cylinder with the gradient across
    its axis, as its cross-section (the three-layer disk): T2 = 40 ms in no
    layer, in the inner one, or in the two outer ones; delta = Delta = 10 ms;
    mixed mode against the oracle."""
    inv = {"none": (0.0, 0.0, 0.0), "inner": (1 / 40000.0, 0.0, 0.0), "outer": (0.0, 1 / 40000.0, 1 / 40000.0)}[t2]
    p = geom.layered_disk(n=24, rho=(1.0, 1.0, 1.0), bvals=(0.0, 2000.0, 4000.0), dirs=((0.0, 1.0, 0.0),))
    p.delta, p.Delta, p.TE = 10000.0, 10000.0, 20000.0
    p.inv_T2 = np.array(inv)
    ref = oracle.run(p)
    sim = sim_cls(p)
    try:
        S, err, stat, st = sim.run(bt.BT_MODE_MIXED)
        assert np.all(stat == 0)
        assert rel(S, ref).max() < TOL_MIXED, rel(S, ref)
    finally:
        sim.close()


def _three_layer(kind):
    """Section 4's three-layer structures (radii 5, 7.5, 10 um; torus ring
    radius 20 um) with per-layer diffusivities 3e-3, 1e-3, 3e-3 and permeable
    membranes; a short PGSE keeps the oracle quick."""
    if kind == "disk":
        p = geom.layered_disk(n=24, D=3e-3, rho=(1.0, 1.0, 1.0), bvals=(1000.0, 4000.0))
        p.D_cmpt = np.array([3e-3, 1e-3, 3e-3])
    elif kind == "sphere":
        p = geom.layered_sphere(n=12)
    else:
        p = geom.layered_torus(h=3.0)
    p.dt, p.delta, p.Delta, p.TE = 50.0, 2500.0, 5000.0, 7500.0
    p.dirs = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]]) if kind != "disk" else np.array([[1.0, 0.0, 0.0]])
    return p


@pytest.mark.parametrize("kind", ["disk", "sphere", "torus"])
def test_three_layer_structures(sim_cls, bt, kind):
    p = _three_layer(kind)
    ref = oracle.run(p)
    sim = sim_cls(p)
    try:
        S, err, stat, st = sim.run(bt.BT_MODE_MIXED)
        assert np.all(stat == 0)
        assert rel(S, ref).max() < TOL_MIXED, rel(S, ref)
    finally:
        sim.close()


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_weak_periodic_projection_on_non_matching_sides(sim_cls, bt, mode):
    """A box whose x sides are sheared against each other: the weak coupling
    reads the opposite side's field at the shifted nodes (projection), against
    the oracle."""
    p = geom.sheared_box(n=5, L=8.0, eps=0.3, bvals=(1000.0, 2500.0),
                         dirs=((1.0, 0.0, 0.0), (0.0, 0.6, 0.8)))
    p.weak_periodic = {"axes": 7, "kappa_e": None}
    ref = oracle.run(p)
    sim = sim_cls(p)
    try:
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S, err, stat, st = sim.run(m)
        assert np.all(stat == 0)
        tol = TOL_FP64 if mode == "plain" else TOL_MIXED
        assert rel(S, ref).max() < tol, rel(S, ref)
    finally:
        sim.close()


def test_batch_of_thin_layers_per_geometry(sim_cls, bt):
    """Three capped spheres of different radii as one uneven batch (surface
    triangles): each geometry's signals against its own oracle run."""
    parts = [geom.spherical_shell(level=2, R=r, kappa=1e-4, cap_z=0.3, bvals=(0.0, 2000.0),
                                  dirs=((1.0, 0.0, 0.0), (0.0, 0.0, 1.0))) for r in (3.0, 4.5, 6.0)]
    u = geom.union(parts)
    ref = np.concatenate([oracle.run(p) for p in parts])
    sim = sim_cls(u)
    try:
        S, err, stat, _ = sim.run(bt.BT_MODE_MIXED)
        assert np.all(stat == 0)
        assert rel(S, ref).max() < TOL_MIXED, rel(S, ref)
    finally:
        sim.close()

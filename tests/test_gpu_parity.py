"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle on
the same seeded inputs.  Tolerances (relative, |S_gpu - S_oracle| / |S_oracle|):
  plain FP64 mode   1e-10
  mixed mode        1e-6   (FP32 Krylov inside double-float refinement)
  assembled planes  1e-13 of the plane's largest entry."""
import json
import math
import os

import numpy as np
import pytest

import geom
import oracle
from oracle import btoracle as bo

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")

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


# ---------------------------------------------------------------- assembly
@pytest.mark.parametrize("maker", [lambda: geom.cfg2(n=8, kappa=1e-3),
                                   lambda: geom.cfg3(n=8, n_dir=2, n_b=1),
                                   lambda: geom.cfg4(n=10, n_dir=1, bvals=(1000.0,))])
def test_assembled_planes_match_oracle(sim_cls, bt, maker):
    p = maker()
    a = bo.assemble(p)
    sim = sim_cls(p)
    try:
        rp, col = bt.bt_get_pattern(sim.ctx)
        for nm in ["M", "K", "J", "MD", "Mx", "My", "Mz", "Ex", "Ey", "Ez"]:
            v = bt.bt_get_plane(sim.ctx, nm)
            ref = a[nm].tocsr()
            # oracle value at every slot of the shared pattern (0 where absent)
            dense = np.zeros_like(v)
            for i in range(len(rp) - 1):
                cols = col[rp[i]:rp[i + 1]]
                row = ref.getrow(i)
                m = dict(zip(row.indices, row.data))
                dense[rp[i]:rp[i + 1]] = [m.get(c, 0.0) for c in cols]
            scale = max(np.abs(dense).max(), 1e-300)
            assert np.abs(v - dense).max() <= 1e-13 * scale, nm
        A0 = bt.bt_get_plane(sim.ctx, "A0")
        M = bt.bt_get_plane(sim.ctx, "M")
        KJ = bt.bt_get_plane(sim.ctx, "K") + bt.bt_get_plane(sim.ctx, "J")
        assert np.abs(A0 - (M + 0.5 * p.dt * KJ)).max() <= 1e-14 * np.abs(A0).max()
    finally:
        sim.close()


# ---------------------------------------------------------------- small live parity
CASES = {
    "cfg1_n8": lambda: geom.cfg1(n=8),
    "cfg2_n8": lambda: geom.cfg2(n=8, kappa=1e-4),
    "cfg2_n8_dirs": lambda: _dirs(geom.cfg2(n=8, kappa=1e-4, bvals=(1000.0, 3000.0))),
    "cfg3_n8": lambda: geom.cfg3(n=8, n_dir=3, n_b=2),
    "cfg4_n10": lambda: geom.cfg4(n=10, n_dir=2, bvals=(500.0, 3000.0)),
}


def _dirs(p):
    d = np.array([[1.0, 0.0, 0.0], [0.2, -0.5, 0.7], [0.0, 0.0, 1.0]])
    p.dirs = d / np.linalg.norm(d, axis=1, keepdims=True)
    return p


@pytest.fixture(scope="module")
def live_ref():
    cache = {}

    def get(name):
        if name not in cache:
            p = CASES[name]()
            cache[name] = (p, oracle.run(p))
        return cache[name]
    return get


@pytest.mark.parametrize("name", list(CASES))
def test_plain_fp64_matches_oracle(sim_cls, bt, live_ref, name):
    p, ref = live_ref(name)
    sim = sim_cls(p)
    try:
        S, err, stat, st = sim.run(bt.BT_MODE_PLAIN_FP64)
        assert np.all(stat == 0)
        assert rel(S, ref).max() < TOL_FP64, (S, ref)
    finally:
        sim.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("resid", ["df", "fp64"])
def test_mixed_matches_oracle(sim_cls, bt, live_ref, name, resid):
    p, ref = live_ref(name)
    sim = sim_cls(p)
    try:
        flags = bt.BT_OPT_RESID_FP64 if resid == "fp64" else 0
        S, err, stat, st = sim.run(bt.BT_MODE_MIXED, flags=flags)
        assert np.all(stat == 0)
        e = rel(S, ref)
        assert e.max() < TOL_MIXED, (e, err)
        # the stated error proxy bounds the observed error
        assert np.all(e <= np.maximum(err, 1e-15) * 10 + 1e-12)
    finally:
        sim.close()


@pytest.fixture(scope="module")
def live_field():
    cache = {}

    def get(name):
        if name not in cache:
            p = CASES[name]()
            cache[name] = (p,) + oracle.run(p, return_field=True)
        return cache[name]
    return get


@pytest.mark.parametrize("name", ["cfg1_n8", "cfg2_n8_dirs", "cfg3_n8", "cfg4_n10"])
@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_field_matches_oracle_elementwise(sim_cls, bt, live_field, name, mode):
    """u^N at TE, every dof of every RHS, against the oracle's field (the two
    number dofs the same way: sorted (master node, compartment) pairs).  The
    bound is on |u - U| per entry relative to max |U| of that RHS."""
    p, ref, U = live_field(name)
    sim = sim_cls(p)
    try:
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S, err, stat, st = sim.run(m)
        assert np.all(stat == 0)
        tol = TOL_FP64 if mode == "plain" else TOL_MIXED
        for r in range(p.n_rhs):
            u = bt.bt_get_state(sim.ctx, r)
            assert u.shape == U[r].shape
            e = np.abs(u - U[r]) / np.abs(U[r]).max()
            assert e.max() < tol, (r, e.max(), int(e.argmax()))
        with pytest.raises(bt.BtError):
            bt.bt_get_state(sim.ctx, p.n_rhs)
    finally:
        sim.close()


@pytest.mark.parametrize("name", ["cfg1_n8", "cfg2_n8_dirs", "cfg3_n8", "cfg4_n10"])
@pytest.mark.parametrize("variant", ["row", "halo"])
@pytest.mark.parametrize("loop", ["graph", "host"])
def test_krylov_variants_match_oracle(sim_cls, bt, live_field, name, variant, loop):
    """Each inner-Krylov variant (row SpMM; halo-staged apply with the fused
    direction and solution updates and halo-staged residuals), driven by
    the captured run graph or by the host loop: signals and fields against
    the oracle at the mixed-mode bound."""
    p, ref, U = live_field(name)
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
            assert (np.abs(u - U[r]) / np.abs(U[r]).max()).max() < TOL_MIXED
        st_ = sim.stats()
        assert st_["sys_iters"] > 0 and st_["sys_iters"] <= st_["spmm_launches"] * p.n_rhs
    finally:
        sim.close()


WINDING = {
    "cube": lambda: geom.cfg1(n=8),
    "sphere": lambda: geom.cfg2(n=8, kappa=1e-4, bvals=(1000.0,)),
}


@pytest.fixture(scope="module")
def winding():
    cache = {}

    def get(name):
        if name not in cache:
            p = WINDING[name]()
            p.dirs = geom.fibonacci_dirs(32)
            cache[name] = (p, np.asarray(oracle.run(p)))
        return cache[name]
    return get


@pytest.mark.parametrize("name", list(WINDING))
@pytest.mark.parametrize("variant", ["row", "halo", "slice"])
def test_mixed_mode_recovers_from_failed_inner_solves(sim_cls, bt, winding, name, variant):
    """32 directions over the full 150-step PGSE sequence (lab frame): for a
    few directions the phase of u winds several times across the box, the
    unconjugated (r, D^-1 r) of COCG nearly cancels and an FP32 inner solve
    stalls far from its tolerance.  The refinement must treat such a pass as
    failed (not as the rounding floor) and restart, so every signal still
    matches the oracle at the mixed-mode bound."""
    p, ref = winding(name)
    flags = {"row": bt.BT_OPT_VARIANT_ROW, "halo": bt.BT_OPT_VARIANT_HALO,
             "slice": bt.BT_OPT_VARIANT_SLICE}[variant]
    sim = sim_cls(p)
    try:
        S, err, stat, _ = sim.run(bt.BT_MODE_MIXED, flags=flags)
        assert np.all(stat == 0)
        e = rel(S, ref)
        assert e.max() < TOL_MIXED, (e.max(), int(e.argmax()), err.max())
        assert np.all(err < 1e-5), err.max()
    finally:
        sim.close()


def test_field_of_rhs_range(sim_cls, bt, live_field):
    """A run over an RHS sub-range returns the fields of exactly those RHS."""
    p, ref, U = live_field("cfg2_n8_dirs")
    sim = sim_cls(p)
    try:
        sim.run(bt.BT_MODE_PLAIN_FP64, rhs_begin=2, rhs_end=4)
        for r in (2, 3):
            u = bt.bt_get_state(sim.ctx, r)
            assert (np.abs(u - U[r]) / np.abs(U[r]).max()).max() < TOL_FP64
        for r in (1, 4):
            with pytest.raises(bt.BtError):
                bt.bt_get_state(sim.ctx, r)
        bt.bt_set_gradients(sim.ctx, p.dirs, p.bvals)      # discards the state
        with pytest.raises(bt.BtError):
            bt.bt_get_state(sim.ctx, 2)
    finally:
        sim.close()


def test_free_periodic_exact_closed_form_gpu(sim_cls, bt):
    """Periodic box without compartments: the exact discrete product (P-5)."""
    p = geom.free_periodic_box(n=10, L=10.0, dirs=((0.3, 0.4, math.sqrt(0.75)), (1.0, 0.0, 0.0)),
                               bvals=(1000.0, 3000.0))
    sim = sim_cls(p)
    try:
        for mode, tol in [(bt.BT_MODE_PLAIN_FP64, 1e-11), (bt.BT_MODE_MIXED, 1e-8)]:
            S, err, stat, st = sim.run(mode)
            _, F = oracle.pgse_tables(p.delta, p.Delta, p.dt, p.n_steps)
            for r in range(p.n_rhs):
                q = float(oracle.q_from_b(p.bvals[r % 2], p.delta, p.Delta))
                prod = np.prod((1 - 0.5 * p.dt * 2e-3 * q * q * F[:-1] ** 2) /
                               (1 + 0.5 * p.dt * 2e-3 * q * q * F[1:] ** 2))
                assert abs(S[r] / 1000.0 - prod) < tol
    finally:
        sim.close()


# ---------------------------------------------------------------- stored oracle signals (full sizes)
def _golden(name):
    path = os.path.join(GOLDEN, name + ".json")
    if not os.path.exists(path):
        pytest.skip(f"golden file {name} not generated")
    with open(path) as f:
        g = json.load(f)
    p = getattr(geom, g["builder"])(**g["kwargs"])
    cnt = np.bincount(p.tet_cmpt, minlength=p.n_cmpt)
    fp = g["fingerprint"]
    assert int(np.sum(np.arange(len(cnt)) * cnt)) == fp["cmpt_weighted_sum"], "seeded geometry differs"
    return p, g


@pytest.mark.parametrize("name", ["cfg1_full", "cfg2_full", "cfg3_n20", "cfg4_n24", "cfg2_n12_dt100"])
@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_golden_signals(sim_cls, bt, name, mode):
    p, g = _golden(name)
    ref = np.array(g["S_re"]) + 1j * np.array(g["S_im"])
    sim = sim_cls(p)
    try:
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S = np.zeros(len(g["rhs"]), complex)
        for k, r in enumerate(g["rhs"]):
            Sk, err, stat, st = sim.run(m, rhs_begin=r, rhs_end=r + 1)
            assert stat[r] == 0
            S[k] = Sk[r]
        tol = TOL_FP64 if mode == "plain" else TOL_MIXED
        assert rel(S, ref).max() < tol, rel(S, ref)
    finally:
        sim.close()


# ---------------------------------------------------------------- arbitrary temporal profiles
def _profile_case(kind):
    p = geom.cfg2(n=6, kappa=1e-4, bvals=(800.0, 2500.0))
    p.dirs = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]])
    p.delta, p.Delta = 1500.0, 2000.0
    p.TE = {"cos_ogse": 0.5 * (1500.0 + 2000.0) + 1500.0, "sin_ogse": 0.5 * (1500.0 + 2000.0) + 1500.0,
            "double_pgse": 2 * 3500.0, "trapezoid": 3500.0}[kind]
    p.profile = {"kind": kind, "n_periods": 2, "ramp": 200.0}
    return p


@pytest.mark.parametrize("kind", ["cos_ogse", "sin_ogse", "double_pgse", "trapezoid"])
@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_profiles_match_oracle(sim_cls, bt, kind, mode):
    """bt_set_waveform (the library's own tables) against the oracle's own
    quadrature of f, lab frame, signals of every RHS."""
    p = _profile_case(kind)
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


def test_free_periodic_profile_exact_gpu(sim_cls, bt):
    """Periodic box, cos-OGSE: the exact discrete product with the profile's F."""
    p = geom.free_periodic_box(n=8, L=8.0, dirs=((0.3, 0.4, math.sqrt(0.75)),), bvals=(600.0, 1500.0))
    p.delta, p.Delta = 2000.0, 2000.0
    p.TE = 0.5 * (p.delta + p.Delta) + p.delta
    p.profile = {"kind": "cos_ogse", "n_periods": 2}
    F, I = bt.bt_waveform_tables("cos_ogse", p.delta, p.Delta, p.TE, p.dt, n_periods=2)
    sim = sim_cls(p)
    try:
        for mode, tol in [(bt.BT_MODE_PLAIN_FP64, 1e-11), (bt.BT_MODE_MIXED, 1e-8)]:
            S, err, stat, st = sim.run(mode)
            for r, b in enumerate(p.bvals):
                q2 = b / I
                prod = np.prod((1 - 0.5 * p.dt * 2e-3 * q2 * F[:-1] ** 2) / (1 + 0.5 * p.dt * 2e-3 * q2 * F[1:] ** 2))
                assert abs(S[r] / 512.0 - prod) < tol
    finally:
        sim.close()


# ---------------------------------------------------------------- relaxation and initial conditions
@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_relaxation_and_initial_condition_match_oracle(sim_cls, bt, mode):
    """Per-compartment 1/T2 and initial magnetization (bt_set_relaxation) with
    permeable membranes and gradients: the relaxation plane against the
    oracle's, then signals and fields against the oracle."""
    p = geom.cfg2(n=6, kappa=1e-4, bvals=(0.0, 1000.0, 2500.0))
    p.dirs = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]])
    p.inv_T2 = np.array([1.0 / 30000.0, 1.0 / 70000.0])
    p.rho = np.array([1.0, 0.55])
    ref, U = oracle.run(p, return_field=True)
    sim = sim_cls(p)
    try:
        a = bo.assemble(p)
        rp, col = bt.bt_get_pattern(sim.ctx)
        v = bt.bt_get_plane(sim.ctx, "MR")
        dense = np.zeros_like(v)
        mr = a["MR"].tocsr()
        for i in range(len(rp) - 1):
            row = mr.getrow(i)
            m = dict(zip(row.indices, row.data))
            dense[rp[i]:rp[i + 1]] = [m.get(c, 0.0) for c in col[rp[i]:rp[i + 1]]]
        assert np.abs(v - dense).max() <= 1e-13 * np.abs(dense).max()
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S, err, stat, st = sim.run(m)
        assert np.all(stat == 0)
        tol = TOL_FP64 if mode == "plain" else TOL_MIXED
        assert rel(S, ref).max() < tol, rel(S, ref)
        for r in range(p.n_rhs):
            u = bt.bt_get_state(sim.ctx, r)
            assert (np.abs(u - U[r]) / np.abs(U[r]).max()).max() < tol
    finally:
        sim.close()


# ---------------------------------------------------------------- anisotropic diffusion
@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_diffusion_tensor_matches_oracle(sim_cls, bt, mode):
    """Per-compartment diffusion tensors (lab frame): the stiffness plane
    against the oracle's, then the signals."""
    p = geom.cfg2(n=6, kappa=1e-4, bvals=(1000.0, 2500.0))
    p.dirs = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]])
    p.D_tensor = np.array([[2.0e-3, 1.1e-3, 0.6e-3, 0.3e-3, -0.2e-3, 0.15e-3],
                           [1.0e-3, 1.5e-3, 2.5e-3, -0.4e-3, 0.35e-3, 0.1e-3]])
    ref = oracle.run(p)
    sim = sim_cls(p)
    try:
        a = bo.assemble(p)
        rp, col = bt.bt_get_pattern(sim.ctx)
        v = bt.bt_get_plane(sim.ctx, "K")
        kk = a["K"].tocsr()
        dense = np.zeros_like(v)
        for i in range(len(rp) - 1):
            row = kk.getrow(i)
            m = dict(zip(row.indices, row.data))
            dense[rp[i]:rp[i + 1]] = [m.get(c, 0.0) for c in col[rp[i]:rp[i + 1]]]
        assert np.abs(v - dense).max() <= 1e-13 * np.abs(dense).max()
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S, err, stat, st = sim.run(m)
        assert np.all(stat == 0)
        tol = TOL_FP64 if mode == "plain" else TOL_MIXED
        assert rel(S, ref).max() < tol, rel(S, ref)
    finally:
        sim.close()


def test_diffusion_tensor_refused_in_transformed_frame(bt):
    p = geom.free_periodic_box(n=3, L=5.0)
    ctx = bt.bt_create(0)
    try:
        bt.bt_upload_mesh(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, 7, p.box_lo, p.box_hi)
        bt.bt_set_diffusion_tensor(ctx, np.array([[2e-3, 1e-3, 1e-3, 0.0, 0.0, 0.0]]))
        with pytest.raises(bt.BtError) as e:
            bt.bt_assemble(ctx, 50.0, 0.5, bt.BT_FRAME_TRANSFORMED)
        assert e.value.code == bt.BT_EINVAL
        with pytest.raises(bt.BtError) as e:
            bt.bt_set_diffusion_tensor(ctx, np.array([[1e-3, 1e-3, 1e-3, 2e-3, 0.0, 0.0]]))  # indefinite
        assert e.value.code == bt.BT_EINVAL
    finally:
        bt.bt_destroy(ctx)


# ---------------------------------------------------------------- weak pseudo-periodic box
def _weak_box(dt=50.0):
    p = geom.free_periodic_box(n=6, L=8.0, dt=dt, bvals=(800.0, 2000.0),
                               dirs=((1.0, 0.0, 0.0), (0.3, 0.4, math.sqrt(0.75))))
    p.periodic_mask = 0
    p.transformed = False
    p.weak_periodic = {"axes": 7, "kappa_e": None}
    return p


def _weak_cells():
    p = geom.cfg2(n=6, kappa=1e-4, bvals=(1000.0, 2500.0))
    p.dirs = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]])
    p.weak_periodic = {"axes": 5, "kappa_e": 4e-3}
    return p


def _weak_square_disk():
    d = (1 / math.sqrt(2), 1 / math.sqrt(2), 0.0)
    p = geom.square_disk(n=12, L=10.0, R=3.0, dt=100.0, kappa=1e-4, bvals=(1000.0, 3000.0), dirs=(d, (1.0, 0, 0)))
    p.delta, p.Delta, p.TE = 10000.0, 13000.0, 23000.0
    p.weak_periodic = {"axes": 3, "kappa_e": None}
    return p


@pytest.mark.parametrize("case", ["box", "cells", "square_disk"])
@pytest.mark.parametrize("mode", ["plain", "mixed", "mixed_host"])
def test_weak_periodic_matches_oracle(sim_cls, bt, case, mode):
    """Artificial-permeability coupling of the box faces (bt_set_weak_periodic)
    against the oracle: a free box coupled on all axes, the sphere case
    coupled on x and z with a given kappa_e, and in 2-D a disk in a square
    coupled through its side edges; captured graph and host loop."""
    p = {"box": _weak_box, "cells": _weak_cells, "square_disk": _weak_square_disk}[case]()
    ref = oracle.run(p)
    sim = sim_cls(p)
    try:
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        flags = bt.BT_OPT_NO_GRAPH if mode == "mixed_host" else 0
        S, err, stat, st = sim.run(m, flags=flags)
        assert np.all(stat == 0)
        tol = TOL_FP64 if mode == "plain" else TOL_MIXED
        assert rel(S, ref).max() < tol, rel(S, ref)
    finally:
        sim.close()


def test_weak_periodic_refusals(bt):
    q = geom.free_periodic_box(n=3, L=5.0)
    ctx = bt.bt_create(0)
    try:
        bt.bt_upload_mesh(ctx, q.xyz, q.tets, q.tet_cmpt, q.D_cmpt, q.kappa_cmpt, 7, q.box_lo, q.box_hi)
        with pytest.raises(bt.BtError) as e:
            bt.bt_set_weak_periodic(ctx, 1, 0.0)              # axis already periodic in the mesh
        assert e.value.code == bt.BT_EINVAL
        bt.bt_upload_mesh(ctx, q.xyz, q.tets, q.tet_cmpt, q.D_cmpt, q.kappa_cmpt, 0, q.box_lo, q.box_hi)
        bt.bt_set_weak_periodic(ctx, 7, 0.0)
        with pytest.raises(bt.BtError) as e:
            bt.bt_assemble(ctx, 50.0, 0.5, bt.BT_FRAME_TRANSFORMED)
        assert e.value.code == bt.BT_EINVAL
    finally:
        bt.bt_destroy(ctx)


# ---------------------------------------------------------------- 2-D triangles
def test_triangle_planes_match_oracle(sim_cls, bt):
    p = geom.square_disk(n=12, L=10.0, R=3.0, kappa=1e-4)
    a = bo.assemble(p)
    sim = sim_cls(p)
    try:
        rp, col = bt.bt_get_pattern(sim.ctx)
        for nm in ["M", "K", "J", "MD", "Mx", "My", "Mz", "Ex", "Ey", "Ez"]:
            v = bt.bt_get_plane(sim.ctx, nm)
            ref = a[nm].tocsr()
            dense = np.zeros_like(v)
            for i in range(len(rp) - 1):
                m = dict(zip(ref.getrow(i).indices, ref.getrow(i).data))
                dense[rp[i]:rp[i + 1]] = [m.get(c, 0.0) for c in col[rp[i]:rp[i + 1]]]
            scale = max(np.abs(dense).max(), 1e-300)
            assert np.abs(v - dense).max() <= 1e-13 * scale, nm
    finally:
        sim.close()


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_triangle_signals_match_oracle(sim_cls, bt, mode):
    """Disk in a square (lab frame), two directions and three b-values."""
    p = geom.square_disk(n=16, L=10.0, R=3.0, kappa=1e-4, bvals=(0.0, 1000.0, 3000.0),
                         dirs=((1.0, 0.0, 0.0), (0.6, 0.8, 0.0)))
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


def test_triangle_periodic_square_exact_product_gpu(sim_cls, bt):
    """Free diffusion in a periodic square (transformed frame): the exact
    discrete product of the theta-scheme."""
    p = geom.free_periodic_square(n=8, L=6.0, dt=50.0, dirs=((0.6, 0.8, 0.0), (1.0, 0.0, 0.0)),
                                  bvals=(900.0, 2000.0))
    sim = sim_cls(p)
    try:
        fbar, F, I = oracle.sequence(p)
        for mode, tol in [(bt.BT_MODE_PLAIN_FP64, 1e-11), (bt.BT_MODE_MIXED, 1e-8)]:
            S, err, stat, st = sim.run(mode)
            assert np.all(stat == 0)
            for r in range(p.n_rhs):
                q2 = p.bvals[r % 2] / I
                prod = np.prod((1 - 0.5 * p.dt * 2e-3 * q2 * F[:-1] ** 2) / (1 + 0.5 * p.dt * 2e-3 * q2 * F[1:] ** 2))
                assert abs(S[r] / 36.0 - prod) < tol
    finally:
        sim.close()


def test_triangle_directions_must_lie_in_plane(sim_cls, bt):
    p = geom.square_disk(n=4, L=10.0, R=3.0, dirs=((0.6, 0.0, 0.8),))
    with pytest.raises(bt.BtError) as e:
        sim_cls(p)
    assert e.value.code == bt.BT_EINVAL


# ---------------------------------------------------------------- 1-D manifolds
def _tree():
    return geom.dendrite_tree(seed=4, n_stems=4, depth=4, length=(10.0, 25.0))


def test_manifold_planes_match_oracle(sim_cls, bt):
    p = _tree()
    a = bo.assemble(p)
    sim = sim_cls(p)
    try:
        rp, col = bt.bt_get_pattern(sim.ctx)
        for nm in ["M", "K", "J", "MD", "Mx", "My", "Mz", "Ex", "Ey", "Ez"]:
            v = bt.bt_get_plane(sim.ctx, nm)
            ref = a[nm].tocsr()
            dense = np.zeros_like(v)
            for i in range(len(rp) - 1):
                m = dict(zip(ref.getrow(i).indices, ref.getrow(i).data))
                dense[rp[i]:rp[i + 1]] = [m.get(c, 0.0) for c in col[rp[i]:rp[i + 1]]]
            scale = max(np.abs(dense).max(), 1e-300)
            assert np.abs(v - dense).max() <= 1e-13 * scale, nm
    finally:
        sim.close()


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_manifold_signals_match_oracle(sim_cls, bt, mode):
    """Branched dendrite tree, three directions and three b-values."""
    p = _tree()
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


def test_manifold_transformed_frame_refused(bt):
    p = geom.line_segments(8)
    ctx = bt.bt_create(0)
    try:
        bt.bt_upload_mesh_1d(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.box_lo, p.box_hi)
        with pytest.raises(bt.BtError) as e:
            bt.bt_assemble(ctx, 50.0, 0.5, bt.BT_FRAME_TRANSFORMED)
        assert e.value.code == bt.BT_EINVAL
        bt.bt_assemble(ctx, 50.0, 0.5, bt.BT_FRAME_LAB)
    finally:
        bt.bt_destroy(ctx)


# ---------------------------------------------------------------- thin layers (surfaces in 3-D)
def _shell():
    return geom.spherical_shell(level=3, R=5.0, kappa=1e-4, cap_z=0.3, bvals=(0.0, 1000.0, 3000.0),
                                dirs=((1.0, 0.0, 0.0), (0.3, -0.5, 0.8)))


def test_surface_planes_match_oracle(sim_cls, bt):
    p = _shell()
    a = bo.assemble(p)
    sim = sim_cls(p)
    try:
        rp, col = bt.bt_get_pattern(sim.ctx)
        for nm in ["M", "K", "J", "MD", "Mx", "My", "Mz", "Ex", "Ey", "Ez"]:
            v = bt.bt_get_plane(sim.ctx, nm)
            ref = a[nm].tocsr()
            dense = np.zeros_like(v)
            for i in range(len(rp) - 1):
                m = dict(zip(ref.getrow(i).indices, ref.getrow(i).data))
                dense[rp[i]:rp[i + 1]] = [m.get(c, 0.0) for c in col[rp[i]:rp[i + 1]]]
            scale = max(np.abs(dense).max(), 1e-300)
            assert np.abs(v - dense).max() <= 1e-13 * scale, nm
    finally:
        sim.close()


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_surface_signals_match_oracle(sim_cls, bt, mode):
    """Sphere with a permeable cap, two 3-D directions and three b-values."""
    p = _shell()
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


def test_surface_transformed_frame_refused(bt):
    p = geom.spherical_shell(level=1)
    ctx = bt.bt_create(0)
    try:
        bt.bt_upload_mesh_surface(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, p.box_lo, p.box_hi)
        with pytest.raises(bt.BtError) as e:
            bt.bt_assemble(ctx, 50.0, 0.5, bt.BT_FRAME_TRANSFORMED)
        assert e.value.code == bt.BT_EINVAL
        bt.bt_assemble(ctx, 50.0, 0.5, bt.BT_FRAME_LAB)
    finally:
        bt.bt_destroy(ctx)

"""The slice-tiled Krylov iteration (variant 2: Morton tiles with a 32-system
slice of p staged in shared memory, then an r update with the inner products
and an x/p update) against the FP64 oracle, for
every vector layout it serves (1, 2 and 4 right-hand sides per lane), both
frames (COCG in the lab frame, CG in the transformed frame), both drivers
(captured run graph, host loop), all five configurations (tiles of 256 or
128 halo rows; two pipelined shared-memory stages or one; one, two or three
blocks per SM; a copy warp feeding fifteen summing warps) and an uneven batch.  Bound: mixed mode,
1e-6 relative per signal, and every dof of every field at 1e-6 of its
largest value."""
import numpy as np
import pytest

import geom
import oracle

pytestmark = pytest.mark.gpu

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


def _short(p, delta, Delta):
    p.delta, p.Delta, p.TE = delta, Delta, delta + Delta
    return p


def _nb1_lab():
    p = geom.cfg2(n=8, kappa=1e-4, bvals=(1000.0,))
    p.dirs = geom.fibonacci_dirs(32)  # 32 RHS, one b-value: one system per lane
    return p


CASES = {
    # 32 directions x 4 b-values = 128 RHS: four systems per lane (COCG)
    "nb4_lab": lambda: _short(geom.cfg4(n=8, n_dir=32, bvals=(500.0, 1000.0, 2000.0, 3000.0)), 1000.0, 2000.0),
    # 16 directions x 4 b-values = 64 RHS: two per lane, periodic box (CG)
    "nb2_transformed": lambda: _short(geom.cfg3(n=6, n_dir=16, n_b=4), 500.0, 1000.0),
    # 32 directions x 1 b-value: one per lane
    "nb1_lab": _nb1_lab,
}


@pytest.fixture(scope="module")
def field():
    cache = {}

    def get(name):
        if name not in cache:
            p = CASES[name]()
            cache[name] = (p,) + oracle.run(p, return_field=True)
        return cache[name]
    return get


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("loop", ["graph", "host"])
@pytest.mark.parametrize("cfg", [0, 1, 2, 3, 4])
def test_slice_variant_matches_oracle(sim_cls, bt, field, name, loop, cfg):
    p, ref, U = field(name)
    flags = bt.slice_config_flag(cfg) | (bt.BT_OPT_NO_GRAPH if loop == "host" else 0)
    sim = sim_cls(p)
    try:
        S, err, stat, _ = sim.run(bt.BT_MODE_MIXED, flags=flags)
        assert np.all(stat == 0)
        e = np.abs(S - ref) / np.abs(ref)
        assert e.max() < TOL_MIXED, e
        for r in range(p.n_rhs):
            u = bt.bt_get_state(sim.ctx, r)
            assert (np.abs(u - U[r]) / np.abs(U[r]).max()).max() < TOL_MIXED, r
        st = sim.stats()
        assert st["krylov_iters"] > 0 and 0 < st["sys_iters"] <= st["spmm_launches"] * p.n_rhs
        tu = bt.bt_get_tuning(sim.ctx)
        assert tu["variant"] == bt.VARIANTS[2 + cfg]
        assert all(tu[f"ms_iter_{v}"] > 0 for v in bt.VARIANTS[2:])
    finally:
        sim.close()


def test_slice_variant_iterations_match_row_variant(sim_cls, bt, field):
    """Both variants run the same Jacobi COCG recurrences, so the iteration
    counts of the same solves differ by a few per cent at most (rounding)."""
    p, ref, U = field("nb4_lab")
    sim = sim_cls(p)
    try:
        sim.run(bt.BT_MODE_MIXED, flags=bt.BT_OPT_VARIANT_ROW | bt.BT_OPT_NO_GRAPH)
        it_row = sim.stats()["sys_iters"]
        sim.run(bt.BT_MODE_MIXED, flags=bt.BT_OPT_VARIANT_SLICE | bt.BT_OPT_NO_GRAPH)
        it_sl = sim.stats()["sys_iters"]
        assert abs(it_sl - it_row) <= 0.05 * it_row, (it_row, it_sl)
    finally:
        sim.close()


def test_slice_variant_in_an_uneven_batch(sim_cls, bt):
    """Two packings of different sizes and PGSE timings as one segmented
    system (tile blocks planned per segment), 64 RHS each, against the
    oracle per geometry."""
    a = _short(geom.cfg4(n=6, n_dir=16, bvals=(500.0, 1000.0, 2000.0, 3000.0), seed=3), 500.0, 1000.0)
    b = _short(geom.cfg4(n=9, n_dir=16, bvals=(500.0, 1000.0, 2000.0, 3000.0), seed=4), 1000.0, 1500.0)
    parts = [a, b]
    ref = np.concatenate([np.asarray(oracle.run(q)) for q in parts])
    sim = sim_cls(geom.union(parts))
    try:
        S, err, stat, _ = sim.run(bt.BT_MODE_MIXED, flags=bt.BT_OPT_VARIANT_SLICE)
        assert np.all(stat == 0)
        assert bt.bt_get_tuning(sim.ctx)["ms_iter_slice"] > 0
        e = np.abs(S - ref) / np.abs(ref)
        assert e.max() < TOL_MIXED, e
    finally:
        sim.close()


def test_slice_flag_falls_back_when_the_width_does_not_fit(sim_cls, bt):
    """One RHS (padded width 1): the slice iteration is not offered and the
    flag leaves the tuned choice in place."""
    p = geom.cfg1(n=6)
    ref = oracle.run(p)
    sim = sim_cls(p)
    try:
        S, err, stat, _ = sim.run(bt.BT_MODE_MIXED, flags=bt.BT_OPT_VARIANT_SLICE)
        assert np.all(stat == 0)
        assert np.abs(S - ref).max() / np.abs(ref).max() < TOL_MIXED
        tu = bt.bt_get_tuning(sim.ctx)
        assert tu["variant"] not in bt.VARIANTS[2:]
        assert all(tu[f"ms_iter_{v}"] == 0 for v in bt.VARIANTS[2:])
    finally:
        sim.close()

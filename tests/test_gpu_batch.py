"""The uneven batch: several geometries with their own PGSE timing solved as
one segmented system.  Each geometry's signals must equal those of the oracle
(small union) or of separate single-geometry GPU runs (seeded packings)."""
import numpy as np
import pytest

import geom
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    from paper_1908_01719_gb300 import build, bt as btmod
    build.build()
    return btmod


@pytest.fixture(scope="module")
def sim_cls(bt):
    from paper_1908_01719_gb300.simulate import Simulation
    return Simulation


def _small_union():
    a = geom.cfg1(n=5)
    a.delta, a.Delta, a.TE = 1000.0, 2000.0, 3000.0       # 60 steps
    a.bvals = np.array([800.0, 2500.0])
    b = geom.cfg2(n=6, kappa=1e-4, bvals=(800.0, 2500.0))  # 150 steps
    c = geom.cfg2(n=4, kappa=3e-4, bvals=(800.0, 2500.0))
    c.delta, c.Delta, c.TE = 1500.0, 3000.0, 4500.0       # 90 steps
    return [a, b, c]


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_small_union_matches_oracle_per_geometry(sim_cls, bt, mode):
    parts = _small_union()
    u = geom.union(parts)
    runs = [oracle.run(p, return_field=True) for p in parts]
    ref = np.concatenate([r[0] for r in runs])
    sim = sim_cls(u)
    try:
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S, err, stat, _ = sim.run(m)
        assert len(S) == 3 * 2 and np.all(stat == 0)
        tol = 1e-10 if mode == "plain" else 1e-6
        assert np.max(np.abs(S - ref) / np.abs(ref)) < tol, (S, ref)
        # each segment's field at its own echo time, dof by dof
        for g, (_, U) in enumerate(runs):
            for r in range(2):
                ug = bt.bt_get_state(sim.ctx, g * 2 + r)
                assert ug.shape == U[r].shape
                assert np.max(np.abs(ug - U[r])) / np.abs(U[r]).max() < tol, (g, r)
    finally:
        sim.close()


def test_seeded_packings_batch_equals_separate_runs(sim_cls, bt):
    parts = [geom.cfg5_geometry(g, scale=0.2, n_dir=4, bvals=(1000.0, 3000.0)) for g in range(4)]
    u = geom.union(parts)
    sim = sim_cls(u)
    try:
        S, err, stat, _ = sim.run(bt.BT_MODE_MIXED)
        assert np.all(stat == 0)
    finally:
        sim.close()
    R = 8
    for g, p in enumerate(parts):
        s1 = sim_cls(p)
        try:
            Sg, _, st, _ = s1.run(bt.BT_MODE_MIXED)
        finally:
            s1.close()
        assert np.all(st == 0)
        assert np.max(np.abs(S[g * R:(g + 1) * R] - Sg) / np.abs(Sg)) < 1e-6, g


def test_segment_stats_add_up(sim_cls, bt):
    """Per-geometry SpMM counts (bt_get_segment_stats) sum to the run's total
    and are larger for a geometry with a longer sequence (more time steps)."""
    parts = _small_union()
    u = geom.union(parts)
    sim = sim_cls(u)
    try:
        sim.run(bt.BT_MODE_MIXED)
        seg = bt.bt_get_segment_stats(sim.ctx, 3)
        st = sim.stats()
        assert seg.sum() == st["sys_iters"] and np.all(seg > 0)
        assert seg[1] > seg[0]          # 150 steps against 60
        with pytest.raises(bt.BtError):
            bt.bt_get_segment_stats(sim.ctx, 2)
    finally:
        sim.close()

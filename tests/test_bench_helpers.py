"""The benchmark's pure helpers (no GPU): the algorithmic byte model of the
dominant kernel, the workload description and the oracle sample sizing."""
import numpy as np

import bench
import geom


def test_spmm_bytes_model():
    n, nnz = 1000, 15000
    # one launch, lab frame (4 planes), two vectors per active system (row SpMM)
    matrix = 4 * (n + 1) + nnz * (4 + 16)
    assert bench.spmm_bytes(n, nnz, False, 1, [0], [n], 2) == matrix
    assert bench.spmm_bytes(n, nnz, False, 1, [3], [n], 2) == matrix + 3 * 2 * n * 8
    # the transformed frame reads one more plane (MD)
    assert bench.spmm_bytes(n, nnz, True, 1, [0], [n], 2) == 4 * (n + 1) + nnz * (4 + 20)
    # six vectors per active system (halo apply), two launches
    assert bench.spmm_bytes(n, nnz, False, 2, [5], [n], 6) == 2 * matrix + 5 * 6 * n * 8
    # an uneven batch: each system spans its own geometry's rows
    assert bench.spmm_bytes(n, nnz, False, 1, [4, 1], [900, 100], 6) == matrix + (4 * 900 + 1 * 100) * 6 * 8
    assert bench.VECTORS_PER_SYSTEM["slice1"] == 2 and bench.VECTORS_PER_ITER["slice1"] == 10


def test_segment_rows_of_a_batch():
    """Rows per geometry from the library's dof map (host-only context)."""
    from paper_1908_01719_gb300.simulate import Simulation
    parts = [geom.cfg1(n=3), geom.cfg2(n=4, kappa=1e-4, bvals=(1000.0,))]
    for q in parts:
        q.dirs, q.bvals = parts[0].dirs, parts[0].bvals
    u = geom.union(parts)
    sim = Simulation(u, device=-1)
    try:
        rows = bench.segment_rows(sim, u)
        singles = []
        for q in parts:
            s1 = Simulation(q, device=-1)
            singles.append(s1.n_dof)
            s1.close()
        assert rows.tolist() == singles and rows.sum() == sim.n_dof
    finally:
        sim.close()


def test_step_units_of_an_uneven_batch():
    """Each geometry of a batch counts its own time steps."""
    a, b = geom.cfg1(n=3), geom.cfg1(n=3)
    b.delta, b.Delta, b.TE = 1000.0, 2000.0, 3000.0
    u = geom.union([a, b])
    assert bench.step_units(u) == u.n_rhs * (a.n_steps + b.n_steps)
    assert bench.step_units(a) == a.n_steps * a.n_rhs and bench.step_units(u, 2) == 2 * (a.n_steps + b.n_steps)


def test_describe_and_batch_counts():
    p = geom.cfg1(n=4)
    d = bench.describe("cfg1", p, 125, 1000, 0)
    assert d["rhs"] == 1 and d["time_steps"] == p.n_steps and "Kuhn tets" in d["workload"]
    trees = geom.union([geom.dendrite_tree(seed=s, n_stems=1, depth=1, length=(3.0, 5.0)) for s in range(3)])
    assert bench.n_geometries(trees) == 3 and bench.n_geometries(p) == 1
    d = bench.describe("trees1d", trees, len(trees.xyz), 10, 0)
    assert d["rhs"] == 3 * trees.n_rhs and "segments (1-D manifold)" in d["workload"]
    assert "3 geometries as one uneven batch" in d["workload"]


def test_workloads_and_oracle_samples():
    p = bench.disk2d(n=8)
    assert p.tets.shape[1] == 3 and p.n_rhs == 128
    assert np.allclose(p.dirs[:, 2], 0.0) and np.allclose(np.linalg.norm(p.dirs, axis=1), 1.0)
    assert bench.oracle_grid("cfg4") == bench.ORACLE_GRID and bench.oracle_grid("disk2d") == 192


def test_every_krylov_variant_has_a_byte_model():
    """The bench reports the roofline of whichever variant the library used:
    every name bt_get_tuning can return needs its vector counts and kernel."""
    from paper_1908_01719_gb300 import bt
    for v in bt.VARIANTS:
        assert v in bench.VECTORS_PER_SYSTEM and v in bench.VECTORS_PER_ITER and v in bench.KERNEL, v
    assert bt.slice_config_flag(0) == 1 << bt.BT_OPT_SLICE_CONFIG_SHIFT
    assert len(bt.VARIANTS) == 2 + 5

"""The benchmark's pure helpers (no GPU): the algorithmic byte model of the
dominant kernel, the workload description and the oracle sample sizing."""
import numpy as np

import bench
import geom


def test_spmm_bytes_model():
    n, nnz = 1000, 15000
    # one launch, lab frame (4 planes), row variant (2 vectors per active system)
    matrix = 4 * (n + 1) + nnz * (4 + 16)
    assert bench.spmm_bytes(n, nnz, False, 1, 0, "row") == matrix
    assert bench.spmm_bytes(n, nnz, False, 1, 3, "row") == matrix + 3 * 2 * n * 8
    # the transformed frame reads one more plane (MD)
    assert bench.spmm_bytes(n, nnz, True, 1, 0, "row") == 4 * (n + 1) + nnz * (4 + 20)
    # the halo apply moves six vectors per active system
    assert bench.spmm_bytes(n, nnz, False, 2, 5, "halo") == 2 * matrix + 5 * 6 * n * 8
    # an uneven batch: a system spans its own geometry's rows, n / G on average
    assert bench.spmm_bytes(n, nnz, False, 1, 4, "halo", G=4) == matrix + 4 * 6 * (n / 4) * 8


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

"""The multi-GPU path on CPU: two gloo ranks each solve their share of the
right-hand sides (with the CPU oracle standing in for a GPU) and gather the
signals; the result must equal the unsharded solve exactly.  Also the
partition helpers."""
import os
import socket

import numpy as np

from paper_1908_01719_gb300 import shard


def test_rhs_partition_covers_everything_once():
    for R, world, align in [(128, 2, 4), (128, 3, 4), (5, 2, 1), (512, 8, 8), (7, 4, 1)]:
        got = [shard.rhs_partition(R, world, r, align) for r in range(world)]
        assert got[0][0] == 0 and got[-1][1] == R
        for (a0, a1), (b0, b1) in zip(got, got[1:]):
            assert a1 == b0
        sizes = [b - a for a, b in got]
        assert max(sizes) - min(sizes) <= align
        assert all(a % align == 0 for a, _ in got)


def test_geometry_partition_balances():
    rng = np.random.default_rng(0)
    costs = np.exp(rng.uniform(np.log(5e4), np.log(2e6), 32))
    parts = shard.geometry_partition(costs, 4)
    assert sorted(sum(parts, [])) == list(range(32))
    loads = [costs[p].sum() for p in parts]
    assert max(loads) <= sum(costs) / 4 + costs.max()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import geom
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = geom.cfg2(n=5, kappa=1e-4, bvals=(500.0, 1500.0, 3000.0))
    p.dirs = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]])
    b0, b1 = shard.rhs_partition(p.n_rhs, world, rank, align=len(p.bvals))
    local = oracle.run(p, rhs=range(b0, b1))
    full = shard.gather_signals(local, np.arange(b0, b1), p.n_rhs)
    dist.destroy_process_group()
    q.put((rank, full))


def test_two_gloo_ranks_gather_equals_unsharded():
    import multiprocessing as mp

    import geom
    import oracle
    ctx = mp.get_context("spawn")
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):    # one BLAS thread per rank
        os.environ.setdefault(k, "1")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = geom.cfg2(n=5, kappa=1e-4, bvals=(500.0, 1500.0, 3000.0))
    p.dirs = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]])
    ref = oracle.run(p)
    for r in (0, 1):
        assert np.array_equal(res[r], ref)


def _forest():
    import geom
    return [geom.dendrite_tree(seed=s, n_stems=2, depth=2, length=(6.0, 12.0), bvals=(1000.0,), n_dir=2)
            for s in range(5)]


def _forest_worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    trees = _forest()
    R = trees[0].n_rhs
    mine = shard.geometry_partition([len(t.tets) for t in trees], world)[rank]
    local = [oracle.run(trees[g]) for g in mine]
    index = [g * R + r for g in mine for r in range(R)]
    full = shard.gather_signals(np.concatenate(local) if local else np.zeros(0, complex), index, len(trees) * R)
    dist.destroy_process_group()
    q.put((rank, mine, full))


def test_two_gloo_ranks_shard_a_forest_by_geometry():
    """A batch of dendrite trees (1-D manifolds) split across two ranks by
    geometry (LPT on segment counts), no exchange but the final gather: every
    rank ends with the unsharded batch's signals, bit for bit."""
    import multiprocessing as mp

    import oracle
    ctx = mp.get_context("spawn")
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_forest_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in procs:
        rank, mine, full = q.get(timeout=300)
        res[rank] = (mine, full)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert sorted(res[0][0] + res[1][0]) == list(range(5)) and res[0][0] and res[1][0]
    ref = np.concatenate([oracle.run(t) for t in _forest()])
    for r in (0, 1):
        assert np.array_equal(res[r][1], ref)

"""Multi-GPU sharding of independent units: right-hand sides of one geometry
or whole geometries of a batch.  Units never exchange data inside the time
loop, so each rank (one process per GPU) solves its own share and the only
communication is a host-side gather of the signals at the end (a few complex
numbers per unit).  torch.distributed is the transport (NCCL or gloo)."""
from __future__ import annotations

import numpy as np


def rhs_partition(R: int, world: int, rank: int, align: int = 1):
    """Contiguous RHS range [begin, end) of `rank`: blocks of `align` RHS (a
    direction's b-values stay together) dealt as evenly as possible."""
    if R % align:
        raise ValueError("R must be a multiple of align")
    blocks = R // align
    base, extra = divmod(blocks, world)
    b0 = rank * base + min(rank, extra)
    b1 = b0 + base + (1 if rank < extra else 0)
    return b0 * align, b1 * align


def geometry_partition(costs, world: int):
    """Longest-processing-time assignment of geometries (cost ~ nodes x RHS x
    steps) to ranks; returns one sorted list of geometry indices per rank."""
    order = np.argsort(-np.asarray(costs, dtype=np.float64), kind="stable")
    load = np.zeros(world)
    parts = [[] for _ in range(world)]
    for g in order:
        r = int(np.argmin(load))
        parts[r].append(int(g))
        load[r] += costs[g]
    return [sorted(p) for p in parts]


def gather_signals(local, index, n_total: int, group=None):
    """All ranks' (index, signal) pairs assembled into the full complex signal
    vector of length n_total (on every rank)."""
    import torch
    import torch.distributed as dist
    payload = (np.asarray(index, dtype=np.int64), np.asarray(local, dtype=np.complex128))
    world = dist.get_world_size(group)
    got = [None] * world
    dist.all_gather_object(got, payload, group=group)
    out = np.full(n_total, np.nan + 0j)
    for idx, val in got:
        out[idx] = val
    _ = torch  # transport only
    return out

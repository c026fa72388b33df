"""Write the stored oracle signals used by the GPU parity tests.

Calls only ``geom`` (inputs) and ``oracle`` (the CPU FP64 solve); nothing here
touches the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py [name ...]

Each case is a seeded workload (full size where the sparse direct solve is
feasible, otherwise a reduced grid of the same seeded geometry) and a sample of
its right-hand sides.  The file records the geometry fingerprint so that a
test can tell a changed input from a changed result.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import geom  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    # name: (builder, kwargs, rhs sample or None for all)
    "cfg1_full": ("cfg1", {}, None),
    "cfg2_full": ("cfg2", {}, None),
    "cfg3_n20": ("cfg3", {"n": 20}, [0, 7, 8 * 21 + 3, 8 * 42 + 5, 8 * 63 + 7]),
    "cfg4_n24": ("cfg4", {"n": 24}, [3, 4 * 9 + 1, 4 * 17 + 2, 4 * 31 + 3]),
    "cfg2_n12_dt100": ("cfg2", {"n": 12, "dt": 100.0}, None),
}


def fingerprint(p):
    cnt = np.bincount(p.tet_cmpt, minlength=p.n_cmpt)
    return {"n_nodes": int(len(p.xyz)), "n_tets": int(len(p.tets)),
            "cmpt_counts_head": [int(x) for x in cnt[:8]],
            "cmpt_weighted_sum": int(np.sum(np.arange(len(cnt)) * cnt)),
            "n_cmpt": int(p.n_cmpt)}


def build(name):
    b, kw, _ = CASES[name]
    return getattr(geom, b)(**kw)


def _work(args):
    name, r = args
    import oracle
    p = build(name)
    t0 = time.time()
    S = oracle.run(p, rhs=[r])[0]
    return name, r, complex(S), time.time() - t0


def main(names):
    tasks = []
    for nm in names:
        p = build(nm)
        rhs = CASES[nm][2]
        rhs = list(range(p.n_rhs)) if rhs is None else rhs
        tasks += [(nm, r) for r in rhs]
    ctx = mp.get_context("spawn")
    res = {}
    with ctx.Pool(min(len(tasks), int(os.environ.get("GOLDEN_PROCS", "6")))) as pool:
        for nm, r, S, dt in pool.imap_unordered(_work, tasks):
            res.setdefault(nm, {})[r] = (S, dt)
            print(f"{nm} rhs {r}: S = {S:.15g}  ({dt:.1f} s)", flush=True)
    for nm in names:
        p = build(nm)
        rs = sorted(res[nm])
        out = {"case": nm, "builder": CASES[nm][0], "kwargs": CASES[nm][1],
               "fingerprint": fingerprint(p), "rhs": rs,
               "S_re": [res[nm][r][0].real for r in rs], "S_im": [res[nm][r][0].imag for r in rs],
               "oracle_seconds": [res[nm][r][1] for r in rs],
               "producer": "tests/golden/make_golden.py (oracle.run, splu per step matrix)"}
        with open(os.path.join(HERE, nm + ".json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))

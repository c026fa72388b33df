"""One small, short run of a workload for profilers (ncu): the seeded geometry
of a config on a chosen grid, a shortened PGSE sequence (a few time steps),
mixed precision.  It prints the sizes and the counters of the run.

  python profile_case.py --config cfg4 --grid 64 --steps 2 [--variant halo]

--config disk2d takes --grid as the cells per side of the disk-in-square (32
in-plane directions x 4 b-values); --config trees1d takes it as the number of
dendrite trees in the batch.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import geom
    from paper_1908_01719_gb300 import bt
    from paper_1908_01719_gb300.build import build
    from paper_1908_01719_gb300.simulate import Simulation

    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="cfg4", choices=["cfg1", "cfg2", "cfg3", "cfg4", "disk2d", "trees1d"])
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--steps", type=int, default=2, help="time steps (pulse on throughout)")
    ap.add_argument("--mode", default="mixed", choices=["mixed", "plain"])
    ap.add_argument("--variant", default="auto", choices=["auto", "row", "halo", "slice", "slice1", "slice_small", "slice_small1", "slice_ws"],
                    help="inner Krylov variant (auto: the autotuner's choice)")
    a = ap.parse_args()
    build()
    if a.config == "disk2d":
        import numpy as np
        ang = np.pi * np.arange(32) / 32
        dirs = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], axis=1)
        p = geom.square_disk(n=a.grid, L=20.0, R=5.0, kappa=1e-4, bvals=(500.0, 1000.0, 2000.0, 3000.0), dirs=dirs)
    elif a.config == "trees1d":
        p = geom.union([geom.dendrite_tree(seed=s) for s in range(a.grid)], name="trees1d")
    else:
        p = getattr(geom, a.config)(n=a.grid)
    # a sequence of `steps` steps: first pulse for half, second for the rest
    half = max(1, a.steps // 2)
    p.delta = half * p.dt
    p.Delta = half * p.dt
    p.TE = 2 * half * p.dt
    seg = getattr(p, "segments", None)
    if seg is not None:
        seg["delta"][:], seg["Delta"][:], seg["TE"][:] = p.delta, p.Delta, p.TE
    sim = Simulation(p)
    mode = bt.BT_MODE_MIXED if a.mode == "mixed" else bt.BT_MODE_PLAIN_FP64
    forced = {"auto": 0, "row": bt.BT_OPT_VARIANT_ROW, "halo": bt.BT_OPT_VARIANT_HALO}
    for c, name in enumerate(bt.VARIANTS[2:]):  # the slice configurations
        forced[name] = bt.slice_config_flag(c)
    flags = bt.BT_OPT_NO_GRAPH | bt.BT_OPT_PROFILE | forced[a.variant]
    S, err, stat, _ = sim.run(mode, flags=flags)
    tuning = bt.bt_get_tuning(sim.ctx) if mode != bt.BT_MODE_PLAIN_FP64 else None
    st = sim.stats()
    print(f"per launch: SpMM-class {st['spmm_ms'] / max(1, st['spmm_launches']):.3f} ms, "
          f"residual {st['resid_ms'] / max(1, st['resid_launches']):.3f} ms")
    print(f"{a.config} grid {a.grid}: n_dof {sim.n_dof}, nnz {sim.nnz}, RHS {sim.R}, stats {sim.stats()}, "
          f"tuning {tuning}")
    sim.close()


if __name__ == "__main__":
    main()

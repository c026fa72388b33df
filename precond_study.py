"""Training and gain study of the learned polynomial preconditioner on the
seeded packing of the default workload (40 um box, 96^3 Kuhn grid, 200 cells,
32 directions x 4 b-values, PGSE delta 2.5 ms / Delta 5 ms).

1. Collect training samples from the method's own step solves at each time
   step size (default dt = 20, 50, 100 us): seeded random time steps of the
   mixed-precision run, every RHS of each (bt_collect_precond_data).
2. Train the network on them (bt_train_precond); hold out a seeded tenth.
3. Fit the fixed Chebyshev polynomial's interval to the same training samples
   (bt_fit_chebyshev), and solve for the best single fixed polynomial.
4. At each dt, run the whole simulation four ways and report wall seconds,
   Krylov iterations and SpMM launches (Krylov SpMMs + Horner SpMMs):
   Jacobi on the row-SpMM host loop (the kernels the polynomial modes use),
   Jacobi as the library tunes it (slice SpMM, CUDA graphs), the learned
   polynomial, and the fixed Chebyshev polynomial.

  python precond_study.py [--grid 96] [--dt 20 50 100] [--samples 10240]
                          [--out weights.json] [--report report.json]

The weights file holds the trained network and the fitted Chebyshev interval;
bench.py loads the one committed in the package (data/precond_cfg4_96.json).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WEIGHTS = os.path.join(ROOT, "paper_1908_01719_gb300", "data", "precond_cfg4_96.json")
# relative accuracy of the collected G and h (FP32 Krylov vectors, FP64 sums)
REL_ERR = 1e-6


def sample_steps(n_steps, k, rng):
    """k distinct seeded time steps (1-based, ascending)."""
    k = min(k, n_steps)
    return np.sort(rng.choice(np.arange(1, n_steps + 1), size=k, replace=False)).astype(np.int32)


def loss_of(c, G, h):
    """Per-sample loss 1 - 2 c.h + c.G c for one fixed c [9] or per-sample c [n][9]."""
    c = np.broadcast_to(c, h.shape)
    return 1.0 - 2.0 * np.sum(c * h, 1) + np.einsum("si,sij,sj->s", c, G, c)


def loss_spread(c, G, h, rel_err):
    """Uncertainty of the per-sample loss for data known to relative accuracy
    rel_err: rel_err (2 |c|.|h| + |c|.|G| |c|), mean over the samples."""
    c = np.abs(np.broadcast_to(c, h.shape))
    return float(np.mean(rel_err * (2.0 * np.sum(c * np.abs(h), 1) + np.einsum("si,sij,sj->s", c, np.abs(G), c))))


def best_fixed(G, h):
    """The single c minimising the mean loss: mean(G) c = mean(h) (least squares)."""
    c, *_ = np.linalg.lstsq(G.mean(0), h.mean(0), rcond=1e-14)
    return c


def per_sample_optimum(G, h):
    """Mean of min_c L_s(c) = 1 - h.G^-1 h, the bound no network can pass."""
    out = []
    for g, v in zip(G, h):
        c, *_ = np.linalg.lstsq(g, v, rcond=1e-14)
        out.append(1.0 - v @ c)
    return float(np.mean(out))


def load_weights(path=WEIGHTS):
    """(network weights, Chebyshev coefficients, provenance) of a weights file."""
    from paper_1908_01719_gb300 import bt
    with open(path) as f:
        d = json.load(f)
    w = np.asarray(d["weights"], dtype=np.float32)
    return w, bt.bt_chebyshev_poly(d["chebyshev"]["lo"], d["chebyshev"]["hi"]), d


def run_modes(sim, bt, weights, cheb, modes=("jacobi_row", "jacobi_tuned", "learned", "chebyshev"), ref=None):
    """One whole simulation per mode, wall-clock timed (bt_run returns after
    the signals are on the host); returns {mode: counters} and the signals.
    Signal differences are taken against `ref`, else the jacobi_tuned run."""
    out, sig = {}, {}
    for m in modes:
        flags = 0
        mode = bt.BT_MODE_MIXED
        if m == "jacobi_row":
            flags = bt.BT_OPT_VARIANT_ROW | bt.BT_OPT_NO_GRAPH
        elif m == "learned":
            mode = bt.BT_MODE_LEARNED
            bt.bt_set_precond_poly(sim.ctx, None)
            bt.bt_load_precond(sim.ctx, weights)
        elif m == "chebyshev":
            mode = bt.BT_MODE_LEARNED
            bt.bt_set_precond_poly(sim.ctx, cheb)
        t0 = time.perf_counter()
        S, err, stat, _ = sim.run(mode, flags=flags, raise_on_status=False)
        secs = time.perf_counter() - t0
        print(f"  {m}: {secs:.1f} s", flush=True)
        st = sim.stats()
        hor = bt.bt_get_precond_stats(sim.ctx)["horner_launches"]
        out[m] = {"seconds": secs, "krylov_iters": st["krylov_iters"], "refine_passes": st["refine_passes"],
                  "spmm_launches": st["spmm_launches"], "horner_launches": hor,
                  "spmm_total": st["spmm_launches"] + hor, "sys_iters": st["sys_iters"],
                  "kernel_launches": st["kernel_launches"], "status_ok": bool(np.all(stat == 0)),
                  "err_est_max": float(np.max(err))}
        sig[m] = np.array(S, copy=True)
        if m == "chebyshev":
            bt.bt_set_precond_poly(sim.ctx, None)
    if ref is None:
        ref = sig.get("jacobi_tuned", next(iter(sig.values())))
    for m in out:
        out[m]["max_rel_diff_vs_jacobi"] = float(np.max(np.abs(sig[m] - ref) / np.abs(ref)))
    return out, sig


def main():
    import geom
    from paper_1908_01719_gb300 import bt
    from paper_1908_01719_gb300.build import build
    from paper_1908_01719_gb300.simulate import Simulation

    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=96)
    ap.add_argument("--dt", type=float, nargs="+", default=[20.0, 50.0, 100.0])
    ap.add_argument("--samples", type=int, default=10240, help="step solves (one per RHS per sampled step)")
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", default=None, help="weights file to write (JSON)")
    ap.add_argument("--report", default=None, help="report file to write (JSON)")
    ap.add_argument("--no-gain", action="store_true", help="skip the whole-simulation comparison")
    a = ap.parse_args()
    build()
    rng = np.random.default_rng(a.seed)
    R = 128
    per_dt = int(np.ceil(a.samples / (R * len(a.dt))))
    feats, Gs, hs, tags = [], [], [], []
    t_collect = {}
    for dt in a.dt:
        p = geom.cfg4(n=a.grid, dt=dt)
        sim = Simulation(p)
        try:
            steps = sample_steps(p.n_steps, per_dt, rng)
            t0 = time.perf_counter()
            f, G, h = bt.bt_collect_precond_data(sim.ctx, steps, p.n_rhs)
            t_collect[str(dt)] = time.perf_counter() - t0
        finally:
            sim.close()
        ok = np.abs(G).sum(axis=(1, 2)) > 0
        feats.append(f[ok])
        Gs.append(G[ok])
        hs.append(h[ok])
        tags += [dt] * int(ok.sum())
        print(f"dt {dt}: {int(ok.sum())} samples from steps {steps.tolist()} in {t_collect[str(dt)]:.1f} s",
              flush=True)
    feat, G, h = np.concatenate(feats), np.concatenate(Gs), np.concatenate(hs)
    n = len(feat)
    perm = rng.permutation(n)
    n_hold = n // 10
    hold, train = perm[:n_hold], perm[n_hold:]

    p0 = geom.cfg4(n=8)  # a small context holds the network while it trains
    s0 = Simulation(p0)
    t0 = time.perf_counter()
    hist = bt.bt_train_precond(s0.ctx, feat[train], G[train], h[train],
                               bt.bt_train_default_opts(epochs=a.epochs, batch=a.batch, seed=a.seed,
                                                        rel_err=REL_ERR))
    t_train = time.perf_counter() - t0
    w = bt.bt_save_precond(s0.ctx)
    coef_tr, loss_tr, _ = bt.bt_precond_eval(s0.ctx, feat[train], G[train], h[train])
    _, loss_ho, _ = bt.bt_precond_eval(s0.ctx, feat[hold], G[hold], h[hold])
    s0.close()
    lo, hi, cheb, loss_cheb_tr = bt.bt_fit_chebyshev(G[train], h[train], rel_err=REL_ERR)
    c_fix = best_fixed(G[train], h[train])
    e0 = np.eye(9)[0]
    Gt, ht, Gh, hh = G[train], h[train], G[hold], h[hold]
    losses = {
        "jacobi": {"train": float(loss_of(e0, Gt, ht).mean()), "heldout": float(loss_of(e0, Gh, hh).mean())},
        "chebyshev": {"train": float(loss_cheb_tr), "heldout": float(loss_of(cheb, Gh, hh).mean()),
                      "uncertainty": loss_spread(cheb, Gt, ht, REL_ERR), "interval": [lo, hi]},
        "best_fixed_polynomial": {"train": float(loss_of(c_fix, Gt, ht).mean()),
                                  "heldout": float(loss_of(c_fix, Gh, hh).mean()),
                                  "uncertainty": loss_spread(c_fix, Gt, ht, REL_ERR)},
        "learned": {"train": float(loss_tr), "heldout": float(loss_ho),
                    "uncertainty": loss_spread(coef_tr, Gt, ht, REL_ERR)},
        "per_sample_optimum": {"train": per_sample_optimum(Gt, ht), "heldout": per_sample_optimum(Gh, hh)},
        "note": f"mean of 1 - 2 c.h + c.G c; uncertainty = its rounding spread for data known to {REL_ERR:g} "
                "relative (FP32 Krylov vectors): a loss below its uncertainty is not resolved by the data",
    }
    print(json.dumps(losses), flush=True)
    report = {"workload": f"cfg4 packing on a {a.grid}^3 Kuhn grid, 32 directions x 4 b-values",
              "samples": {"total": n, "train": len(train), "heldout": n_hold,
                          "per_dt": {str(dt): tags.count(dt) for dt in a.dt}},
              "collect_seconds": t_collect, "train_seconds": t_train, "epochs": a.epochs, "batch": a.batch,
              "loss_first_last_epoch": [float(hist[0]), float(hist[-1])], "mean_loss": losses}
    if a.out:
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        with open(a.out, "w") as fo:
            json.dump({"weights": [float(x) for x in w], "chebyshev": {"lo": lo, "hi": hi},
                       "trained_on": {k: report[k] for k in ("workload", "samples", "epochs", "batch")}
                       | {"dt_us": a.dt, "seed": a.seed}}, fo)
    if a.report:
        with open(a.report, "w") as fo:
            json.dump(report, fo, indent=1)
    if not a.no_gain:
        gain = {}
        for dt in a.dt:
            p = geom.cfg4(n=a.grid, dt=dt)
            sim = Simulation(p)
            try:
                sim.run()  # warm-up: the autotuner's timings and the captured graphs
                res, _ = run_modes(sim, bt, w, cheb)
            finally:
                sim.close()
            units = p.n_steps * p.n_rhs
            for m in res:
                res[m]["step_rhs_per_s"] = units / res[m]["seconds"]
            gain[str(dt)] = res
            report["gain"] = gain
            print(f"dt {dt}: " + json.dumps(res), flush=True)
            if a.report:  # written after each dt, so a cut-off run keeps what it measured
                with open(a.report, "w") as fo:
                    json.dump(report, fo, indent=1)
    if a.report:
        with open(a.report, "w") as fo:
            json.dump(report, fo, indent=1)
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()

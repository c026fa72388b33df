"""Benchmark: Bloch-Torrey step-RHS/s and the fused SpMM's HBM fraction on
GB300, at <= 1e-6 signal error against FP64.

One bench step = one complete simulation of the workload: every time step from
u^0 = 1 to TE for every right-hand side (direction x b-value), ending with the
signals.  value = (time steps x RHS x ranks) / (max over ranks of the timed
wall time).  Default workload: cfg4 (40 um box, 96^3 Kuhn grid, packed spheres
and finite cylinders with per-cell permeability, 32 directions x 4 b-values,
PGSE delta 2.5 ms / Delta 5 ms, dt 50 us, 150 steps), mixed precision (FP32
complex SpMM and COCG inside double-float iterative refinement).

Other workloads (--config): cfg1-cfg3 (the smaller 3-D cases), disk2d (2-D P1
triangles: a disk of radius 5 um in a 20 um square, 512^2 cells, 32 in-plane
directions x 4 b-values) and trees1d (1-D manifolds: 64 seeded dendrite trees
as one uneven batch, PGSE delta 10.6 ms / Delta 43.1 ms, dt 100 us, 3
directions x 3 b-values per tree) and shells (thin layers: 32 capped spheres of
seeded radii as level-5 icospheres, 3 directions x 3 b-values each).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config NAME]
  torchrun --nproc-per-node N bench.py --gpus N ...     (one replica per rank,
                                                        weak scaling, no collective
                                                        on the data path)
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# the oracle's bounded sample: the same seeded geometry on a 24^3 Kuhn grid
# (1/64 of the 96^3 dofs), 8 RHS x all time steps, about 20 s per RHS on one core
ORACLE_GRID = 24
THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
METRIC = "Bloch-Torrey step-RHS/s and HBM %peak, at <=1e-6 signal err vs FP64"
UNIT = "step-RHS/s"


N_TREES = 64
N_SHELLS = 32
# the uneven batch of 32 seeded packings (16 directions x 4 b-values each,
# mixed PGSE timings), at full size or with every grid halved per axis
CFG5_SCALE = {"cfg5": 1.0, "cfg5_half_grid": 0.5}
CFG5_ORACLE_CELLS, CFG5_ORACLE_RHS = 8, 2


def shells(n=N_SHELLS):
    """Thin layers: n spheres of seeded radii U(3, 8) um, level-5 icospheres,
    each with a permeable cap above z = 0.3 R; 3 axis directions x 3 b-values."""
    import geom
    rng = np.random.default_rng(0)
    return [geom.spherical_shell(level=5, R=float(r), kappa=1e-4, cap_z=0.3, bvals=(0.0, 1000.0, 3000.0),
                                 dirs=((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)))
            for r in rng.uniform(3.0, 8.0, n)]


def disk2d(n=512):
    import geom
    ang = np.pi * np.arange(32) / 32
    dirs = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], axis=1)
    return geom.square_disk(n=n, L=20.0, R=5.0, kappa=1e-4, bvals=(500.0, 1000.0, 2000.0, 3000.0), dirs=dirs)


def workload(name):
    import geom
    if name == "disk2d":
        return disk2d()
    if name == "trees1d":
        return geom.union([geom.dendrite_tree(seed=s) for s in range(N_TREES)], name="trees1d")
    if name == "shells":
        return geom.union(shells(), name="shells")
    if name == "cfg4":
        return geom.cfg4()
    if name in CFG5_SCALE:
        return geom.cfg5(scale=CFG5_SCALE[name])
    if name == "cfg3":
        return geom.cfg3()
    if name == "cfg2":
        return geom.cfg2()
    if name == "cfg1":
        return geom.cfg1()
    raise ValueError(name)


def step_units(p, n_rhs=None):
    """Time steps x right-hand sides of one simulation: in an uneven batch each
    geometry runs its own number of steps (TE_g / dt) for its right-hand sides."""
    r = p.n_rhs if n_rhs is None else n_rhs
    seg = getattr(p, "segments", None)
    if seg is None:
        return p.n_steps * r
    return r * int(sum(int(round(te / p.dt)) for te in seg["TE"]))


def geom_mod():
    import geom
    return geom


def n_geometries(p):
    seg = getattr(p, "segments", None)
    return 1 if seg is None else len(seg["node_off"]) - 1


def describe(name, p, n_dof, nnz, n_face):
    elem = {4: "Kuhn tets", 3: "triangles (2-D)", 2: "segments (1-D manifold)"}[p.tets.shape[1]]
    if getattr(p, "surface", False):
        elem = "surface triangles (thin layers)"
    G = n_geometries(p)
    seg = getattr(p, "segments", None)
    steps = (f"{p.n_steps} steps" if seg is None else
             f"{min(int(round(t / p.dt)) for t in seg['TE'])}-{max(int(round(t / p.dt)) for t in seg['TE'])} "
             f"steps per geometry (own PGSE timing each)")
    return {"workload": f"{name}: {len(p.xyz)} nodes, {len(p.tets)} {elem}, {p.n_cmpt} compartments, "
                        + (f"{G} geometries as one uneven batch, " if G > 1 else "") +
                        f"{n_dof} dofs after interface doubling, {nnz} nonzeros, {n_face} interface faces; "
                        f"{len(p.dirs)} dirs x {len(p.bvals)} b-values = {p.n_rhs} RHS; PGSE delta {p.delta/1e3} ms "
                        f"Delta {p.Delta/1e3} ms, dt {p.dt} us, {steps}; "
                        f"{'transformed (periodic)' if p.transformed else 'lab'} frame",
            "n_dof": n_dof, "nnz": nnz, "rhs": p.n_rhs * G, "time_steps": p.n_steps if seg is None else None,
            "step_rhs_per_simulation": step_units(p),
            "l2_policy": "inputs larger than L2: Krylov vectors n_dof x RHS x 8 B each "
                         f"({n_dof * p.n_rhs * 8 / 1e9:.2f} GB) vs 129 MB L2"}


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, dev):
        self.dev = dev
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx = float(c[2])
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle CPU baseline
def _oracle_task(args):
    name, grid, r = args
    import geom
    import oracle
    t0 = time.time()
    if name in CFG5_SCALE:                 # geometry r of the batch on a coarse grid, a few RHS
        p = geom.cfg5_geometry(r, scale=1.0)
        p = geom.cfg5_geometry(r, scale=CFG5_ORACLE_CELLS / p.meta["N"])
        oracle.run(p, rhs=list(range(CFG5_ORACLE_RHS)))
        return time.time() - t0, p.n_steps * CFG5_ORACLE_RHS
    if name in ("trees1d", "shells"):      # one whole geometry (all its RHS) per task
        p = geom.dendrite_tree(seed=r) if name == "trees1d" else shells(r + 1)[r]
        oracle.run(p)
        return time.time() - t0, p.n_steps * p.n_rhs
    p = disk2d(n=grid) if name == "disk2d" else \
        {"cfg4": geom.cfg4, "cfg3": geom.cfg3, "cfg2": geom.cfg2, "cfg1": geom.cfg1}[name](n=grid)
    oracle.run(p, rhs=[r])
    return time.time() - t0, p.n_steps


def oracle_grid(name):
    return {"disk2d": 192, "trees1d": 0, "shells": 0}.get(name, ORACLE_GRID)


def oracle_sample(name, n_rhs_sample, grid):
    """The oracle as it stands on `n_rhs_sample` RHS of the same seeded
    geometry on a coarser grid (3-D: `grid`^3 Kuhn cells; 2-D: `grid`^2
    cells), one process per RHS (spawn pool); for the dendrite trees, the
    first `n_rhs_sample` trees of the batch with all their RHS."""
    cores = min(n_rhs_sample, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    # one BLAS/OpenMP thread per worker: several workers with multi-threaded
    # BLAS under SuperLU oversubscribe the cores and can stall for minutes
    saved = {k: os.environ.get(k) for k in THREAD_VARS}
    os.environ.update({k: "1" for k in THREAD_VARS})
    t0 = time.time()
    try:
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_task, [(name, grid, r) for r in range(n_rhs_sample)])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    wall = time.time() - t0
    units = sum(r[1] for r in res)
    if name in CFG5_SCALE:
        what = (f"{name}: geometries 0..{n_rhs_sample - 1} of the batch, each on a {CFG5_ORACLE_CELLS}^3 Kuhn grid of "
                f"its own box, {CFG5_ORACLE_RHS} RHS each over their own full PGSE sequences")
    elif name in ("trees1d", "shells"):
        what = f"{name}: the first {n_rhs_sample} geometries of the batch, all 9 RHS x {res[0][1] // 9} steps"
    elif name == "disk2d":
        what = f"disk2d seeded geometry on a {grid}^2 grid, {n_rhs_sample} RHS x {res[0][1]} steps"
    else:
        what = f"{name} seeded geometry on a {grid}^3 Kuhn grid, {n_rhs_sample} RHS x {res[0][1]} steps"
    return {"value": units / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": what + f", one process per task, wall {wall:.1f} s including assembly and process start"}


# ---------------------------------------------------------------- main arms
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on a bounded sample of the
    same workload (same metric and unit); rank 0 only."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    sample_rhs, grid = min(16, os.cpu_count() or 1), oracle_grid(args.config)
    vals, walls = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.time()
        r = oracle_sample(args.config, sample_rhs, grid)
        if i >= args.warmup:
            vals.append(r)
            walls.append(time.time() - t0)
    v = float(np.mean([r["value"] for r in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.config, "sample": vals[0]["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# vectors of n complex FP32 values (8 B) each active right-hand side moves per
# launch of the dominant kernel: the row SpMM reads X and writes Y; the
# halo-staged apply reads z, p_prev and x and writes x, p and q; the
# slice-tiled SpMM reads p and writes q
VECTORS_PER_SYSTEM = {"row": 2, "halo": 6, "slice": 2, "slice1": 2, "slice_small": 2, "slice_small1": 2, "slice_ws": 2}
# ... and per Krylov iteration (all launches of one iteration): row 2 + 6 + 3,
# halo 6 + 3 (z update: reads z, q, writes z), slice 2 + 3 (r, q read, r
# written) + 5 (x, p, r read, x, p written)
VECTORS_PER_ITER = {"row": 11, "halo": 9, "slice": 10, "slice1": 10, "slice_small": 10, "slice_small1": 10,
                    "slice_ws": 10}
KERNEL = {"row": "k_spmm_krylov", "halo": "k_spmm_halo",
          "slice": "k_spmm_slice (256-halo-row tiles, two stages, one block per SM)",
          "slice1": "k_spmm_slice (256-halo-row tiles, one stage, two blocks per SM)",
          "slice_small": "k_spmm_slice (128-halo-row tiles, two stages, two blocks per SM)",
          "slice_small1": "k_spmm_slice (128-halo-row tiles, one stage, three blocks per SM)",
          "slice_ws": "k_spmm_slice_ws (256-halo-row tiles, two stages filled by a copy warp, 15 summing warps)"}


# DRAM bytes (read + write) of one launch of the row SpMM k_spmm_krylov<4>, lab
# frame, 128 RHS, measured with ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# on the cfg4 geometry at 64^3 (343,793 dofs); see
# profiles/k_spmm_krylov_cfg4_grid64.md.  The row kernel reads every column
# whatever the number of active systems, so the figure scales with the dofs.
ROW_SPMM_TRAFFIC = {"n_dof": 343793, "bytes": 791.9e6 + 329.7e6}
# the same for the slice SpMM (large tiles, one stage, two blocks per SM),
# captured on a launch with all 128 systems active
SLICE1_SPMM_TRAFFIC = {"n_dof": 343793, "bytes": 482.844672e6 + 314.620416e6, "active": 128}


def spmm_bytes(n, nnz, transformed, launches, seg_iters, seg_rows, vectors):
    """Algorithmic HBM bytes of a kernel summed over its launches: per launch
    the row pointers, column indices and packed FP32 planes (A0 and three
    direction planes, plus MD in the transformed frame), and per active system
    of each launch its vectors (`vectors` x rows x 8 B).  A system spans its
    own geometry's rows: seg_iters[g] (active systems of segment g summed over
    the launches) times seg_rows[g]."""
    planes = 5 if transformed else 4
    matrix = 4 * (n + 1) + nnz * (4 + 4 * planes)
    return launches * matrix + vectors * 8 * float(np.dot(np.asarray(seg_iters, float), np.asarray(seg_rows, float)))


def segment_rows(sim, p):
    """Rows (dofs) of each geometry of the context."""
    seg = getattr(p, "segments", None)
    if seg is None:
        return np.array([sim.n_dof])
    from paper_1908_01719_gb300 import bt
    node, _ = bt.bt_get_dofmap(sim.ctx)
    g_of = np.searchsorted(np.asarray(seg["node_off"]), node, side="right") - 1
    return np.bincount(g_of, minlength=len(seg["node_off"]) - 1)


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1908_01719_gb300 import bt
    from paper_1908_01719_gb300.build import build
    from paper_1908_01719_gb300.simulate import Simulation
    build()

    p = workload(args.config)
    stream = torch.cuda.current_stream(dev)
    t_setup = time.time()
    sim = Simulation(p, device=local, stream=stream.cuda_stream)
    torch.cuda.synchronize(dev)
    t_setup = time.time() - t_setup
    mode = bt.BT_MODE_MIXED
    G = n_geometries(p)
    units = step_units(p)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        sim.run(mode)
    # timed region
    flags = bt.BT_OPT_PROFILE
    spmm_ms, vec_ms, spmm_launch, launches, iters, sys_iters = 0.0, 0.0, 0, 0, 0, 0
    seg_iters = np.zeros(G, dtype=np.int64)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(args.steps):
            S, err, stat, _ = sim.run(mode, flags=flags)
            st = sim.stats()
            spmm_ms += st["spmm_ms"]
            vec_ms += st["vec_ms"]
            spmm_launch += st["spmm_launches"]
            launches += st["kernel_launches"]
            iters += st["krylov_iters"]
            sys_iters += st["sys_iters"]
            seg_iters += bt.bt_get_segment_stats(sim.ctx, G)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    tuning = bt.bt_get_tuning(sim.ctx)
    # the same runs as one captured CUDA graph per simulation (no per-launch
    # events), on at most two simulations to bound the bench's wall time
    n_graph = min(args.steps, 2)
    eg0, eg1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eg0.record(stream)
    for _ in range(n_graph):
        sim.run(mode)
    eg1.record(stream)
    torch.cuda.synchronize(dev)
    ms_graph = eg0.elapsed_time(eg1) * args.steps / n_graph
    ms_t = torch.tensor([ms], device=dev)
    if ws > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = units * args.steps * ws / (ms_max / 1e3)

    # accuracy and the plain per-direction FP64 GPU solve on a sample of RHS;
    # a small uneven batch runs every RHS of every geometry at once, the large
    # one (cfg5) runs single geometries of the batch one RHS at a time
    fp64_ms, fp64_units, errs, fp64_what = 0.0, 0, [], None
    if args.config in CFG5_SCALE:
        sample = []
        for g in (0, 1):  # two seeded geometries of the batch, three RHS each
            pg = geom_mod().cfg5_geometry(g, scale=CFG5_SCALE[args.config])
            sg = Simulation(pg, device=local, stream=stream.cuda_stream)
            try:
                for r in (0, pg.n_rhs // 2, pg.n_rhs - 1):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    S64, _, _, _ = sg.run(bt.BT_MODE_PLAIN_FP64, rhs_begin=r, rhs_end=r + 1)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    fp64_ms += e0.elapsed_time(e1)
                    fp64_units += pg.n_steps
                    errs.append(abs(S[g * p.n_rhs + r] - S64[r]) / abs(S64[r]))
                    sample.append([g, r])
            finally:
                sg.close()
        fp64_what = "geometries 0 and 1 of the batch run alone, three RHS each, one RHS per run"
    else:
        sample = sorted(set([0, p.n_rhs // 3, (2 * p.n_rhs) // 3, p.n_rhs - 1])) if G == 1 else list(range(p.n_rhs))
        ranges = [(r, r + 1) for r in sample] if G == 1 else [(0, 0)]
        for rb, re in ranges:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S64, _, stat64, _ = sim.run(bt.BT_MODE_PLAIN_FP64, rhs_begin=rb, rhs_end=re)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            fp64_ms += e0.elapsed_time(e1)
            idx = [rb] if G == 1 else range(G * p.n_rhs)
            errs += [abs(S[i] - S64[i]) / abs(S64[i]) for i in idx]
        fp64_units = step_units(p, len(sample))
    fp64_rate = fp64_units / (fp64_ms / 1e3)

    # roofline of the dominant kernel (fused FP32 SpMM), from live CUDA events
    n, nnz, nf = sim.n_dof, sim.nnz, sim.n_iface
    seg_rows = segment_rows(sim, p)
    bytes_total = spmm_bytes(n, nnz, p.transformed, spmm_launch, seg_iters, seg_rows,
                             VECTORS_PER_SYSTEM[tuning["variant"]])
    bytes_launch = bytes_total / max(1, spmm_launch)
    avg_ms = spmm_ms / max(1, spmm_launch)
    achieved = bytes_total / (spmm_ms / 1e3) / 1e9
    # the whole Krylov iteration of the chosen variant over the timed runs:
    # the SpMM launches and the vector kernels of every iteration, timed by
    # CUDA events inside the library; bytes as for the SpMM with the vectors
    # of all launches of an iteration
    v = tuning["variant"]
    planes = 5 if p.transformed else 4
    it_bytes = spmm_bytes(n, nnz, p.transformed, spmm_launch, seg_iters, seg_rows, VECTORS_PER_ITER[v])
    it_ms = spmm_ms + vec_ms
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"

    # the polynomial preconditioners on the same workload: the network trained
    # by precond_study.py (96^3, dt 20/50/100 us) and its fitted fixed
    # Chebyshev polynomial, against Jacobi on the same row-SpMM host loop and
    # against the tuned Jacobi path; one whole simulation each, wall clock
    learned = None
    if args.config == "cfg4" and ws == 1 and not args.no_learned:
        import precond_study as ps
        if os.path.exists(ps.WEIGHTS):
            w, cheb, meta = ps.load_weights()
            modes, _ = ps.run_modes(sim, bt, w, cheb, ref=S)
            for m in modes.values():
                m["step_rhs_per_s"] = units / m["seconds"]
            learned = {"unit": UNIT, "modes": modes, "chebyshev_interval": [meta["chebyshev"]["lo"],
                                                                            meta["chebyshev"]["hi"]],
                       "trained_on": meta["trained_on"],
                       "gain_vs_jacobi_tuned": modes["jacobi_tuned"]["seconds"] / modes["learned"]["seconds"],
                       "gain_vs_chebyshev": modes["chebyshev"]["seconds"] / modes["learned"]["seconds"],
                       "note": "BT_MODE_LEARNED timed as a whole simulation (wall clock, signals on the host); "
                               "spmm_total = Krylov SpMM launches + Horner SpMM launches; gains are time ratios "
                               "(> 1: the learned polynomial is faster)"}
        else:
            learned = {"unavailable": "no trained weights in the package (precond_study.py --out)"}

    # DRAM traffic per launch from one ncu capture of the 64^3 case of the same
    # geometry, scaled to this grid by the dof ratio; for the slice kernel the
    # capture had every system active, so it is set beside the algorithmic
    # bytes at that activity
    traffic, traffic_note = None, "no capture of this kernel on this workload"
    if args.config == "cfg4" and tuning["variant"] == "row":
        traffic = ROW_SPMM_TRAFFIC["bytes"] * n / ROW_SPMM_TRAFFIC["n_dof"]
        traffic_note = "ncu DRAM bytes per launch of the 64^3 case scaled by the dof ratio"
    elif args.config == "cfg4" and tuning["variant"] == "slice1":
        traffic = SLICE1_SPMM_TRAFFIC["bytes"] * n / SLICE1_SPMM_TRAFFIC["n_dof"]
        full = spmm_bytes(n, nnz, p.transformed, 1, [SLICE1_SPMM_TRAFFIC["active"]], [n], 2)
        traffic_note = (f"ncu DRAM bytes of one 64^3 launch with all {SLICE1_SPMM_TRAFFIC['active']} systems "
                        f"active, scaled by the dof ratio; algorithmic bytes at that activity {full:.4g}")

    # end to end through the public API from host buffers
    torch.cuda.synchronize(dev)
    t0 = time.time()
    sim2 = Simulation(p, device=local, stream=stream.cuda_stream)
    S2, err2, stat2, _ = sim2.run(mode)
    torch.cuda.synchronize(dev)
    e2e_s = time.time() - t0
    sim2.close()
    # what the library copies to the device: nodes, elements, compartments and
    # diffusivities; interface faces (element, local vertices, kappa); the
    # element and face contribution lists with their slot pointers; the
    # pattern; per run the directions, q and the sequence tables
    nv = p.tets.shape[1]
    fs = nv - 1
    h2d = (p.xyz.nbytes + 4 * nv * len(p.tets) + 4 * len(p.tets) + p.D_cmpt.nbytes + nf * (4 + fs + 8) +
           8 * (nnz + 1) * 2 + 4 * (nv * nv * len(p.tets) + (2 * fs) ** 2 * nf) + 4 * (n + 1) + 4 * nnz +
           (3 * 8 + 8) * p.n_rhs * G + 48 * p.n_steps * G)
    d2h = p.n_rhs * G * (16 + 8 + 4) + 8 * n
    sim.close()

    if rank != 0:
        return
    cpu = oracle_sample(args.config, min(16, os.cpu_count() or 1), oracle_grid(args.config)) if ws == 1 else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32 (SpMM/Krylov) + double-float residual",
            "data": "synthetic",
            "config": dict(describe(args.config, p, n, nnz, nf),
                           parallelism=f"replica per GPU x{ws}", setup_s=round(t_setup, 2),
                           krylov_iters_per_run=iters / args.steps),
            "accuracy": {"max_rel_err_vs_gpu_fp64": float(max(errs)), "rhs_checked": sample,
                         "err_est_max": float(np.max(err))},
            "fp64_plain_per_direction_gpu": {"value": fp64_rate, "unit": UNIT, "rhs_sample": sample,
                                             "speedup_of_value": value / ws / fp64_rate,
                                             **({"sample_note": fp64_what} if fp64_what else {})},
            "spmm_autotune": tuning,
            "roofline": {"bound": "hbm",
                         "kernel": KERNEL[tuning["variant"]]
                         + " (fused FP32 complex SpMM of the Krylov iteration, the autotuned variant)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_src, "frac_of_nominal_7900_gbs": achieved / 7900.0,
                         "traffic": traffic,
                         "traffic_note": traffic_note,
                         "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": avg_ms,
                         "active_rhs_per_launch": sys_iters / max(1, spmm_launch),
                         "launches": spmm_launch},
            "iteration_roofline": {"variant": v, "ms_per_iteration": it_ms / max(1, spmm_launch),
                                   "bytes_per_iteration": it_bytes / max(1, spmm_launch),
                                   "vectors_per_system": VECTORS_PER_ITER[v],
                                   "achieved": it_bytes / (it_ms / 1e3) / 1e9 if it_ms > 0 else None,
                                   "frac": it_bytes / (it_ms / 1e3) / 1e9 / peak if it_ms > 0 else None,
                                   "unit": "GB/s", "note": "all Krylov iterations of the timed runs: SpMM and "
                                   "vector kernels, CUDA events around each launch"},
            "cpu_baseline": cpu,
            "e2e": {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "seconds": e2e_s,
                    "includes": "host mesh pipeline, upload, assembly, full run, signal read-back"},
            "gpu_launches": int(launches), "clocks": clocks,
            **({"learned_preconditioner": learned} if learned is not None else {}),
            "graph_path": {"value": units * args.steps * ws / (ms_graph / 1e3), "unit": UNIT,
                           "note": "same runs, each simulation one captured CUDA graph with nested conditional "
                                   "WHILE nodes; the headline value uses host-driven launches so that every "
                                   "fused SpMM launch is bracketed by CUDA events for the roofline"}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned / Chebyshev / Jacobi preconditioner comparison (cfg4)")
    ap.add_argument("--config", default="cfg4", choices=["cfg1", "cfg2", "cfg3", "cfg4", "disk2d", "trees1d", "shells"]
                    + list(CFG5_SCALE))
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

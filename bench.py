#!/usr/bin/env python3
"""Benchmark of the parallel event-chain sweep for hard disks on GB300.

One step = one full sweep (Sec. 3.4 steps 1-7: binning, four colour phases of
frame staging and chains, reduction) of the workload, here 1024^2 disks at
packing fraction 0.72 from a square lattice (the paper's large-system shape),
seeded and synthetic.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank advances its own
replica (Philox key (seed, rank)): independent replicas, no data exchange.
"""
import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import ecmc_workloads as W  # noqa: E402

METRIC = ("collision events/s, sweeps/s (N=1M, η=0.72); "
          "batched FP32 vs FP64 at equal P error")
UNIT = "events/s"
# Roofline of the chain kernel (the scope table's measurement row): shared
# memory, against ALGORITHMIC bytes per collision event -- the disks whose
# centres lie in the strip that can hold the first hit, area 2 sigma (sigma +
# lambda0) with lambda0 the measured mean free path, read as FP32 (8 B) or
# FP64 (16 B) coordinates, plus 16 B to read and write the active disk
# (smem_bytes_per_event below).
#
# Counters of the persistent sweep kernel k_sweep_fused<8 lanes per cell,
# FP32 screening, axis chains> that need more than one ncu pass, for both
# placements of the FP64 frame coordinates the autotuner chooses between
# (frame mode 1, global scratch: its choice at N = 1M; frame mode 0, shared
# memory): captured at N = 640,000, eta = 0.72 with the paper's parameters
# (188 x 188 cells, about 8,800 active cells per phase), one launch = one sweep
# (profiles/k_sweep_fused_n640k_paper_params.md); the full-size workload is
# profiled with single-pass metric sets only.  Both scale with the work:
# DRAM bytes with the disks (every cell and its halo are read once per colour
# phase), FP64 warp-instructions with the event-loop iterations.
FUSED_CAPTURE_N = 640000
FUSED_ITERATIONS_CAPTURE = 1524505               # contacts + walls + chain ends per launch
FUSED_CAPTURES = {
    # frame mode: dram__bytes_read.sum + _write.sum, smsp__inst_executed_pipe_fp64.sum,
    # sm__pipe_fp64_cycles_active (% of active cycles)
    1: {"dram_bytes": 24786688 + 492544, "fp64_winst": 5594937, "fp64_pipe_pct": 37.95},
    0: {"dram_bytes": 24617216 + 1792, "fp64_winst": 5594741, "fp64_pipe_pct": 37.01},
}
FUSED_CAPTURE_FRAME_MODE = 1                     # the autotuner's choice at N = 1M
FUSED_DRAM_BYTES_CAPTURE = FUSED_CAPTURES[1]["dram_bytes"]
FUSED_FP64_WINST_CAPTURE = FUSED_CAPTURES[1]["fp64_winst"]
FUSED_NCU_FP64_PIPE_PCT = FUSED_CAPTURES[1]["fp64_pipe_pct"]


def fused_capture(captured):
    """The ncu counters for the run's configuration: a frame mode with a
    capture, True for the autotuner's usual choice, or None."""
    if captured is True:
        return FUSED_CAPTURES[FUSED_CAPTURE_FRAME_MODE]
    if captured is False or captured is None:
        return None
    return FUSED_CAPTURES.get(captured)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["small", "medium", "large", "huge", "batch", "eos"])
    ap.add_argument("--tau", action="store_true",
                    help="autocorrelation time of Psi against n_m and ell (N = 64^2)")
    ap.add_argument("--tau-eta", type=float, default=0.704,
                    help="packing fraction of the --tau experiment")
    ap.add_argument("--tau-max", type=int, default=100000,
                    help="most sweeps per point of the --tau experiment")
    ap.add_argument("--listbias", action="store_true",
                    help="pressure vs n_m with start lists drawn with and without replacement")
    ap.add_argument("--fig3", action="store_true",
                    help="g(r) near contact and P(g(sigma+)) vs n_m: reflecting and rejecting "
                         "boundary rules, start lists with and without replacement")
    ap.add_argument("--stripes", action="store_true",
                    help="striped decomposition of Fig. 3: events/s at N = 256^2, eta = 0.708 "
                         "over stripes x ell, both boundary rules")
    ap.add_argument("--dim3", action="store_true",
                    help="hard spheres in three dimensions: events/s over cells x ell (N = 64^3)")
    ap.add_argument("--gr", action="store_true",
                    help="time the pair-correlation histogram (0.01 sigma bins to 5 sigma) on "
                         "the --workload (default medium: N = 65,536) and on the large one")
    ap.add_argument("--grid", action="store_true",
                    help="parallelisation grid at N = 1M (cells x ell), one JSON line")
    ap.add_argument("--paper-params", action="store_true",
                    help="cells, ell, n_m from the paper's strategy (Sec. 4)")
    ap.add_argument("--autotune", action="store_true", help="tune the launch shape first")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--fmode", type=int, default=-1, help="frame placement 0/1/2 (-1 automatic)")
    ap.add_argument("--dir", default="axis", choices=["axis", "iso"],
                    help="chain directions: alternating axes (default) or isotropic")
    ap.add_argument("--persistent", type=int, default=-1,
                    help="1 one persistent launch per sweep, 0 per-phase launches (-1 default)")
    ap.add_argument("--melt", type=int, default=-1,
                    help="untimed sweeps from the lattice before warm-up (default 20; the "
                         "oracle arms run the same sweeps and reach the same state)")
    ap.add_argument("--fixed-params", action="store_true",
                    help="use the workload table's cells/ell instead of the paper's strategy")
    ap.add_argument("--cells", type=int, default=0, help="cells per side (0 = workload default)")
    ap.add_argument("--ell", type=float, default=0.0, help="chain displacement (0 = default)")
    ap.add_argument("--nm", type=int, default=0, help="chains per cell (0 = eq. nm)")
    ap.add_argument("--n", type=int, default=0,
                    help="disks of the large workload (a perfect square; 0 = 1048576): the "
                         "same packing fraction and seed, e.g. a smaller case for profiling")
    ap.add_argument("--tpc", type=int, default=0, help="lanes per cell (0 = automatic)")
    ap.add_argument("--prec", type=int, default=1, help="1 FP32 screening, 0 FP64 candidates")
    ap.add_argument("--no-flush", action="store_true", help="do not flush L2 between steps")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    return ap.parse_args()


def combine_over_ranks(ms, events, sweeps, device=None):
    """Whole-job figures of independent replicas on several ranks: the
    slowest rank's timed milliseconds, and the events and sweeps of all."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(events), float(sweeps)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return t.item(), n[0].item(), n[1].item()


def replica_key(rank, r=0):
    """Philox key word 1 of replica r on a rank: ranks never share a stream."""
    return r + 100000 * rank


def melt_sweeps(args):
    return 20 if args.melt < 0 else args.melt


def workload(args):
    w = {"small": W.SMALL, "medium": W.MEDIUM, "large": W.LARGE, "huge": W.HUGE,
         "batch": W.LARGE, "eos": W.LARGE}[args.workload]
    if args.n and args.workload == "large":
        w = dataclasses.replace(w, N=args.n, name="N=%d eta=%g" % (args.n, w.eta))
    cells = args.cells or w.cells
    ell = args.ell or w.ell
    return w, cells, ell


def batch_descs(args, rank, reference=False):
    """Replica batch descriptors: the paper's strategy (Sec. 4) picks cells,
    ell and n_m for every replica; every rank runs its own replica keys.  The
    reference arm takes the strategy from the oracle, ours from the
    library (the two give the same choice; tests/test_oracle_strategy.py)."""
    reps = W.replica_batch() if args.workload == "batch" else W.eos_batch()
    out = []
    for d in reps:
        if reference:
            import oracle

            c, ell, nm = oracle.suggest_parameters(d["N"], d["L"], 1.0, 2.0)
            s = {"N": d["N"], "L": d["L"], "sigma": 1.0, "cells_x": c, "cells_y": c, "ell": ell,
                 "n_m": nm}
        else:
            from paper_1409_6948_gb300 import ecmc as E

            s = E.suggest_parameters(d["N"], d["L"], 1.0, 2.0)
        s.update(seed=d["seed"], replica=replica_key(rank, d["replica"]), eta=d["eta"])
        out.append(s)
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; start()
    returns once the first sample is in, so the samples cover the region
    that follows."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
            return
        t_end = time.time() + 3.0
        while time.time() < t_end and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [v.strip() for v in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(w, cells, ell, nm, seconds, melt=0, max_sweeps=1000, dir_mode=0):
    """The oracle, as it stands, single-threaded on this host: the same melt
    sweeps (untimed), then sweeps of the same workload until `seconds` have
    passed."""
    import oracle

    L = w.L
    x, y = W.square_lattice(w.N, L)
    if nm == 0:
        nm = oracle.default_nm(w.N, L, 1.0, cells, cells, ell)
    p = oracle.make_params(w.N, L, 1.0, cells, cells, ell, nm, w.seed, dir_mode=dir_mode)
    oracle.sweeps(p, x, y, 0, melt)
    st = oracle.Stats()
    t0 = time.perf_counter()
    n = 0
    while n < max_sweeps:
        oracle.sweeps(p, x, y, melt + n, 1, stats=st)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": st.events / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d sweeps of the full workload after %d untimed melt sweeps (%.1f s)"
                      % (n, melt, dt),
            "sweeps_per_s": n / dt}


def _oracle_batch_worker(job):
    """One host process of the batch CPU baseline: its share of the replicas,
    one oracle sweep each in turn, until `seconds` have passed."""
    descs, seconds = job
    import oracle

    states = []
    for d in descs:
        x, y = W.square_lattice(d["N"], d["L"])
        p = oracle.make_params(d["N"], d["L"], 1.0, d["cells_x"], d["cells_y"], d["ell"],
                               d["n_m"], d["seed"], d["replica"])
        states.append([p, x, y, 0])
    st = oracle.Stats()
    t0 = time.perf_counter()
    n = 0
    while states and time.perf_counter() - t0 < seconds:
        s = states[n % len(states)]
        oracle.sweeps(s[0], s[1], s[2], s[3], 1, stats=st)
        s[3] += 1
        n += 1
    return st.events, n, time.perf_counter() - t0


def cpu_baseline_batch(descs, seconds):
    """The oracle on the batch's replicas with every host core: independent
    replicas need no communication, so each core (a process started with
    spawn, as the parent already holds a CUDA context) runs its share of the
    replicas, one sweep each in turn, for `seconds`."""
    import multiprocessing as mp

    import oracle

    oracle.lib()  # build once here, not in every worker
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    cores = max(1, min(cores, len(descs)))
    jobs = [(descs[i::cores], seconds) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_batch_worker, jobs)
    events = sum(r[0] for r in res)
    sweeps = sum(r[1] for r in res)
    wall = max(r[2] for r in res)
    return {"value": events / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d replica sweeps on %d processes (replicas in turn, from their "
                      "lattice starts, %.1f s)" % (sweeps, cores, wall)}


def run_grid(args):
    """Parallelisation grid at N = 1024^2, eta = 0.72 (Sec. 4, Figs. 5-6),
    through the library's measured tuner (ecmc_tune_geometry, n_m from eq. nm):
    1. the survey's grid -- cells 8^2 .. 512^2 x ell in {2, 8, 32} sigma --
       with its recipe: 100 warm-up sweeps from the lattice, at least 1 s
       timed per point;
    2. the tuner's own candidates around the paper's strategy (cells / 2 ..
       cells x 2 of ecmc_suggest_parameters, ell from ell*/4 to 4 ell* of
       eq. criterion... ell*/8 .. 4 ell*), once with the same recipe and once with short trials
       (10 warm-up, 10 timed sweeps), to check that the short trials pick
       what the long ones pick.
    Each point reports events/s, sweeps/s, the measured mean free path and the
    criterion's ell* from it; the proxy is the mean square displacement per
    second (ECMC_TUNE_MSD)."""
    import torch

    from paper_1409_6948_gb300 import ecmc as E

    torch.cuda.set_device(0)
    w = W.LARGE
    L = w.L
    lam0 = (W.ETA_HCP - w.eta) / (2 * W.ETA_HCP)
    warm = 100 if args.warmup < 100 else args.warmup
    grid, gbest = E.tune_geometry(w.N, L, W.LARGE_CELL_GRID, W.LARGE_ELL_GRID, seed=w.seed,
                                  warm_sweeps=warm, trial_sweeps=10, min_seconds=1.0,
                                  proxy=E.TUNE_MSD)
    for t in grid:
        n_blocks = t["cells"] ** 2 / 4.0
        t["criterion_ell_eq_lambda0"] = L * lam0 / math.sqrt(n_blocks)
        t["N_over_eta_n"] = w.N / (w.eta * n_blocks)
    sp = E.suggest_parameters(w.N, L, 1.0, 2.0)
    c0 = sp["cells_x"]
    cells = sorted({max(2, 2 * int(round(c0 * f / 2))) for f in (0.5, 0.7071, 1.0, 1.4142, 2.0)})
    ells = [sp["ell"] * f for f in (0.125, 0.25, 0.5, 1.0, 2.0, 4.0)]
    long_t, lbest = E.tune_geometry(w.N, L, cells, ells, seed=w.seed, warm_sweeps=warm,
                                    trial_sweeps=10, min_seconds=1.0, proxy=E.TUNE_MSD)
    short_t, sbest = E.tune_geometry(w.N, L, cells, ells, seed=w.seed, warm_sweeps=10,
                                     trial_sweeps=10, min_seconds=0.0, proxy=E.TUNE_MSD)

    def pick(ts, i):
        t = ts[i]
        return {"cells": t["cells"], "ell": t["ell"], "n_m": t["n_m"],
                "msd_per_s": t["score"], "events_per_s": t["events_per_s"],
                "sweeps_per_s": t["sweeps_per_s"], "lambda0": t["lambda0"],
                "ell_star": t["ell_star"]}

    by = lambda ts, k: max(range(len(ts)), key=lambda i: ts[i][k] if ts[i]["status"] == 0  # noqa
                           else -1.0)
    print(json.dumps({
        "mode": "grid", "workload": w.name, "warm_sweeps": warm, "min_seconds": 1.0,
        "proxy": "mean square displacement per second", "lambda0_eq": lam0,
        "survey_grid": {"points": grid, "best_msd": pick(grid, gbest),
                        "best_events": pick(grid, by(grid, "events_per_s")),
                        "best_sweeps": pick(grid, by(grid, "sweeps_per_s"))},
        "paper_strategy": {"cells": c0, "ell": sp["ell"], "n_m": sp["n_m"]},
        "tuner_candidates": {"cells": cells, "ell": ells, "long": long_t, "short": short_t,
                             "best_long": pick(long_t, lbest), "best_short": pick(short_t, sbest),
                             "agree": lbest == sbest}}))
    return 0


def run_listbias(args):
    """Start lists with and without replacement (Sec. 3.4, Fig. 3 right): the
    chain-estimator pressure against the number n_m of chains per cell for
    N = 256^2 disks at eta = 0.708 (32 x 32 cells, ell = 8 sigma).  Every
    point melts the lattice with 4000 / n_m sweeps and measures over
    8000 / n_m sweeps (the same number of chains for every n_m); error bars
    from batch means.  Both list rules start from the same key, so at n_m = 1,
    where the lists coincide, the runs are identical."""
    import torch

    import paper_1409_6948_gb300 as P
    from paper_1409_6948_gb300 import ecmc as E

    torch.cuda.set_device(0)
    w = W.MEDIUM
    pts = []
    for nm in (1, 2, 4, 8, 16):
        for mode in (E.LIST_WITH_REPL, E.LIST_WITHOUT_REPL):
            g = P.Ecmc(w.N, w.L, 1.0, w.cells, w.cells, w.ell, w.seed)
            g.set_param(E.PARAM_N_CHAINS, nm)
            g.set_param(E.PARAM_LIST_MODE, mode)
            g.sweep(4000 // nm)
            g.reset_stats()
            s = torch.cuda.Stream()
            g.set_stream(s)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            g.sweep(8000 // nm)
            b.record(s)
            torch.cuda.synchronize()
            p, se = g.pressure()
            c = g.counters()
            pts.append({"n_m": nm, "list": "with replacement" if mode == 0 else "shuffled",
                        "betaP_sigma2": p, "stderr": se, "sweeps": 8000 // nm,
                        "events_per_s": c.events / (a.elapsed_time(b) * 1e-3)})
            g.set_stream(None)
            g.close()
    for nm in (1, 2, 4, 8, 16):
        pw = [q for q in pts if q["n_m"] == nm]
        d = pw[1]["betaP_sigma2"] - pw[0]["betaP_sigma2"]
        pw[1]["difference_in_combined_se"] = d / math.hypot(pw[0]["stderr"], pw[1]["stderr"])
    print(json.dumps({"mode": "list_bias", "workload": "N=65536 eta=0.708 cells=32x32 ell=8",
                      "points": pts}))
    return 0


def contact_value(r, g, sigma=1.0, nfit=5):
    """g(sigma+) from a quadratic least-squares fit over the first nfit bins,
    evaluated at sigma (the contact extrapolation of the pressure route)."""
    return float(np.polyfit(r[:nfit] - sigma, g[:nfit], 2)[-1])


def run_fig3(args):
    """The comparison of Sec. 3.4, Fig. 3: pair correlations near contact and
    the pressure read from g(sigma+) (eq. pressure) against the number n_m of
    chains per cell, for N = 256^2 disks at eta = 0.708 in 32 x 32 cells.
    Rules: reflection at walls and frozen disks (PEC-refl, ell = 8 sigma) and
    rejection of the whole chain (PEC-rej, ell = 0.25 sigma: a chain's front
    advances about beta P / rho ~ 11 times its budget, so longer chains
    rarely stay inside an 8.4 sigma cell); each with start lists drawn with
    replacement and shuffled.  Every point starts from one configuration
    melted by the paper's algorithm (2000 sweeps with n_m = 4 and ell = 8
    sigma, or --melt), equilibrates for S / (4 n_m) sweeps and
    measures g(r) every 10 sweeps over S / n_m sweeps, the same number of
    chains for every n_m.  Error bars from 8 batches."""
    import torch

    import paper_1409_6948_gb300 as P
    from paper_1409_6948_gb300 import ecmc as E

    torch.cuda.set_device(0)
    w = W.MEDIUM
    N, L = w.N, w.L
    rho = N / (L * L)
    dr, rmax, nbatch = 0.01, 1.5, 8
    g0 = P.Ecmc(N, L, 1.0, w.cells, w.cells, w.ell, w.seed)
    g0.set_param(E.PARAM_N_CHAINS, 4)
    g0.sweep(2000 if args.melt < 0 else args.melt)
    xy0 = g0.positions().copy()
    t0 = g0.sweep_index()
    g0.close()
    nb = int(round((rmax - 1.0) / dr))
    e0 = 1.0 + dr * np.arange(nb)
    e1 = e0 + dr
    R = 2.0 * (e1**3 - e0**3) / (3.0 * (e1**2 - e0**2))
    norm = N * rho * 2.0 * math.pi * R * dr
    pts = []
    for rule, ell, S in (("reflect", 8.0, 8000), ("reject", 0.25, 32000)):
        for nm in (1, 2, 4, 8, 16):
            for mode in (E.LIST_WITH_REPL, E.LIST_WITHOUT_REPL):
                g = P.Ecmc(N, L, 1.0, w.cells, w.cells, ell, w.seed + 1)
                g.set_param(E.PARAM_N_CHAINS, nm)
                g.set_param(E.PARAM_LIST_MODE, mode)
                if rule == "reject":
                    g.set_param(E.PARAM_BOUNDARY, E.BOUNDARY_REJECT)
                g.set_param(E.PARAM_GR_DR, dr)
                g.set_param(E.PARAM_GR_RMAX, rmax)
                g.set_positions(xy0, t0=t0)
                g.sweep(max(1, S // (4 * nm)))
                g.reset_stats()
                per_batch = max(1, S // nm // nbatch // 10)
                prev = np.zeros(nb)
                prev_n = 0
                gs, ps = [], []
                for _ in range(nbatch):
                    for _ in range(per_batch):
                        g.sweep(10)
                        g.gr_measure()
                    cnt, nmeas = g.gr_counts()
                    cnt = cnt[:nb].astype(float)
                    gb = ((cnt - prev) / (nmeas - prev_n)) / norm
                    prev, prev_n = cnt, nmeas
                    gs.append(gb)
                    gc = contact_value(R, gb)
                    ps.append(rho * (1.0 + 0.5 * math.pi * rho * gc))
                gm = np.mean(gs, 0)
                c = g.counters()
                pt = {"rule": rule, "ell": ell, "n_m": nm,
                      "list": "with replacement" if mode == 0 else "shuffled",
                      "betaP_sigma2_gcontact": float(np.mean(ps)),
                      "stderr": float(np.std(ps, ddof=1) / math.sqrt(nbatch)),
                      "g_contact": contact_value(R, gm),
                      "g_first_bins": [round(float(v), 4) for v in gm[:12]],
                      "sweeps": per_batch * nbatch * 10,
                      "rejected_fraction": c.rejected_chains / max(c.chains, 1)}
                if rule == "reflect":
                    pt["betaP_sigma2_chain"] = g.pressure()[0]
                pts.append(pt)
                g.close()
                print(json.dumps(pt), flush=True)
    for rule in ("reflect", "reject"):
        for nm in (1, 2, 4, 8, 16):
            pw = [q for q in pts if q["n_m"] == nm and q["rule"] == rule]
            d = pw[1]["betaP_sigma2_gcontact"] - pw[0]["betaP_sigma2_gcontact"]
            pw[1]["difference_in_combined_se"] = d / math.hypot(pw[0]["stderr"], pw[1]["stderr"])
    print(json.dumps({"mode": "fig3", "workload": "N=65536 eta=0.708 cells=32x32",
                      "points": pts}))
    return 0


def run_dim3(args):
    """Hard spheres in three dimensions (the generalisation of Sec. 3.4;
    include/ecmc3.h): N = 64^3 spheres at eta = 0.45 (dense liquid) from the
    simple cubic lattice, for a small grid of cells per side and chain
    displacements ell, n_m chosen so that a sweep displaces about every
    sphere once (eq. nm with the mean free path measured at this density).
    Each point melts 30 sweeps and times --steps sweeps with CUDA events on
    the library's stream; --cells and --ell restrict the grid to one value.
    The 3D oracle is timed on a bounded sample of the first point on one
    host core."""
    import torch

    import oracle
    import paper_1409_6948_gb300 as P
    from paper_1409_6948_gb300 import ecmc as E

    torch.cuda.set_device(0)
    N, eta, seed = 262144, 0.45, 7
    L = W.box_side3(N, eta)
    lam0 = 0.06  # mean free path at eta = 0.45 (the points report their own)
    pts = []
    for cells in ((args.cells,) if args.cells else (16, 20, 26, 32)):
        for ell in ((args.ell,) if args.ell else (0.5, 1.0, 2.0)):
            nm = max(1, int(round(N / cells**3 * lam0 / ell)))
            g = P.Ecmc3(N, L, 1.0, cells, ell, seed)
            g.set_param(E.PARAM3_N_CHAINS, nm)
            s = torch.cuda.Stream()
            g.set_stream(s)
            g.sweep(30)
            g.reset_stats()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            g.sweep(args.steps)
            b.record(s)
            g.synchronize()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            c = g.counters()
            iters = c.events + c.wall_hits + c.chains
            # FP64 pipe: 13 algorithmic operations per event-loop iteration
            # (hit test of the first candidate: da, dp, dq, dp^2, dq^2, c^2,
            # sigma^2 - c^2, b - sqrt; update: wall distance, new position,
            # new budget, b - s and its sum), against the peak of 2 FP64
            # lanes/clock/SM x SMs x the clock
            n_sm = torch.cuda.get_device_properties(0).multi_processor_count
            peak = 2 * n_sm * 2070e6 / 1e9
            achieved = 13 * iters / (ms * 1e-3) / 1e9
            pt = {"cells": cells, "ell": ell, "n_m": nm, "sweeps": args.steps,
                  "events_per_s": c.events / (ms * 1e-3), "sweeps_per_s": args.steps / (ms * 1e-3),
                  "ms_per_sweep": ms / args.steps, "events_per_sweep": c.events / args.steps,
                  "mean_free_path": c.sum_disp / max(iters, 1),
                  "betaP_sigma3": g.pressure()[0],
                  "roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved,
                               "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
                               "fp64_ops_per_iteration": 13}}
            pts.append(pt)
            print(json.dumps(pt), flush=True)
            g.set_stream(None)
            g.close()
    # the oracle on the first point's workload, one host core, bounded sample
    cpu = None
    if args.cpu_seconds > 0:
        p0 = pts[0]
        x, y, z = W.cubic_lattice(N, L)
        p = oracle.make_params3(N, L, 1.0, p0["cells"], p0["ell"], p0["n_m"], seed)
        oracle.sweeps3(p, x, y, z, 0, 2)
        t0 = time.perf_counter()
        n = 0
        st = oracle.Stats()
        while time.perf_counter() - t0 < args.cpu_seconds and n < 50:
            oracle.sweeps3(p, x, y, z, 2 + n, 1, stats=st)
            n += 1
        dt = time.perf_counter() - t0
        cpu = {"value": st.events / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
               "sample": "%d sweeps of the first point (%.1f s)" % (n, dt)}
    best = max(pts, key=lambda q: q["events_per_s"])
    print(json.dumps({"mode": "dim3", "workload": "N=262144 (64^3) hard spheres eta=0.45",
                      "best": best, "points": pts, "cpu_baseline": cpu}))
    return 0


def run_stripes(args):
    """The striped decomposition of Fig. 3 (include/ecmc_stripes.h) on the
    Fig. 3 system, N = 256^2 disks at eta = 0.708 from the square lattice:
    stripes S in {16, 32, 64}, chain displacement ell in {1, 8} sigma, n_m per
    stripe chosen so that a sweep displaces about every disk once (N / S
    lambda / ell with the mean free path lambda = 0.05 sigma measured at this
    density), for the rejecting (the paper's) and the reflecting rule.  Each
    point melts 20 sweeps and times --steps sweeps with CUDA events on the
    library's stream.  The oracle (orc_stripe_sweeps) is timed on a bounded
    sample of the first point on one host core."""
    import torch

    import oracle
    import paper_1409_6948_gb300 as P
    from paper_1409_6948_gb300 import ecmc as E

    torch.cuda.set_device(0)
    N, eta, seed, lam = 65536, 0.708, 7, 0.05
    L = W.box_side(N, eta)
    pts = []
    for boundary in (E.BOUNDARY_REJECT, E.BOUNDARY_REFLECT):
        for S in (16, 32, 64):
            for ell in (1.0, 8.0):
                nm = max(1, int(round(N / S * lam / ell)))
                g = P.EcmcStripes(N, L, 1.0, S, ell, seed)
                g.set_param(E.PARAM_STRIPES_N_CHAINS, nm)
                g.set_param(E.PARAM_STRIPES_BOUNDARY, boundary)
                s = torch.cuda.Stream()
                g.set_stream(s)
                g.sweep(20)
                g.reset_stats()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                g.sweep(args.steps)
                b.record(s)
                g.synchronize()
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                c = g.counters()
                pt = {"boundary": "reject" if boundary == E.BOUNDARY_REJECT else "reflect",
                      "stripes": S, "ell": ell, "n_m": nm, "sweeps": args.steps,
                      "events_per_s": c.events / (ms * 1e-3),
                      "sweeps_per_s": args.steps / (ms * 1e-3), "ms_per_sweep": ms / args.steps,
                      "events_per_sweep": c.events / args.steps,
                      "rejected_fraction": c.rejected_chains / max(c.chains, 1),
                      "kernel": "sorted frames" if g.get_param(E.PARAM_STRIPES_KERNEL) == 1
                                else "block-wide scan"}
                pts.append(pt)
                print(json.dumps(pt), flush=True)
                g.set_stream(None)
                g.close()
    cpu = None
    if args.cpu_seconds > 0:
        p0 = pts[0]
        x, y = W.square_lattice(N, L)
        p = oracle.make_params(N, L, 1.0, p0["stripes"], p0["stripes"], p0["ell"], p0["n_m"],
                               seed, boundary=oracle.BOUNDARY_REJECT)
        oracle.stripe_sweeps(p, x, y, 0, 2)
        t0 = time.perf_counter()
        n = 0
        st = oracle.Stats()
        while time.perf_counter() - t0 < args.cpu_seconds and n < 200:
            oracle.stripe_sweeps(p, x, y, 2 + n, 1, stats=st)
            n += 1
        dt = time.perf_counter() - t0
        cpu = {"value": st.events / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
               "sample": "%d sweeps of the first point (%.1f s)" % (n, dt)}
    best = max(pts, key=lambda q: q["events_per_s"])
    print(json.dumps({"mode": "stripes", "workload": "N=65536 (256^2) disks eta=0.708, stripes",
                      "best": best, "points": pts, "cpu_baseline": cpu}))
    return 0


def run_gr(args):
    """The pair-correlation histogram of Sec. 2 (0.01 sigma bins from sigma to 5
    sigma, ordered pairs) on a melted state: CUDA-event time per measurement
    (fixed-point positions, then the pair histogram), pairs binned per second.
    One JSON line per workload."""
    import torch

    import paper_1409_6948_gb300 as P
    from paper_1409_6948_gb300 import ecmc as E

    torch.cuda.set_device(0)
    names = ["medium", "large"] if args.workload == "large" else [args.workload, "large"]
    for name in names:
        w = {"small": W.SMALL, "medium": W.MEDIUM, "large": W.LARGE, "huge": W.HUGE}[name]
        L = w.L
        sp = E.suggest_parameters(w.N, L, 1.0, 2.0) if name in ("large", "huge") else \
            {"cells_x": w.cells, "ell": w.ell, "n_m": 0}
        g = P.Ecmc(w.N, L, 1.0, sp["cells_x"], sp["cells_x"], sp["ell"], w.seed)
        if sp["n_m"]:
            g.set_param(E.PARAM_N_CHAINS, sp["n_m"])
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        g.set_stream(stream)
        g.set_param(E.PARAM_GR_DR, 0.01)
        g.set_param(E.PARAM_GR_RMAX, 5.0)
        g.sweep(melt_sweeps(args))
        g.synchronize()
        for _ in range(args.warmup):
            g.gr_measure()
        g.synchronize()
        g.reset_stats()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            g.gr_measure()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        counts, nm = g.gr_counts()
        pairs = float(counts.sum()) / nm
        print(json.dumps({"mode": "gr", "workload": w.name, "N": w.N,
                          "cells": sp["cells_x"], "bins": int(counts.size), "dr": 0.01,
                          "rmax": 5.0, "measurements": args.steps, "us_per_measurement": 1e3 * ms,
                          "ordered_pairs_per_measurement": pairs,
                          "pairs_per_s": pairs / (ms * 1e-3),
                          "disks_per_s": w.N / (ms * 1e-3)}), flush=True)
        g.set_stream(None)
        g.close()
    return 0


def run_tau(args):
    """Sampling efficiency (Sec. 2 eq. tau; Figs. 5-6): the autocorrelation
    time tau of the hexatic order parameter Psi for N = 64^2 disks at
    eta = --tau-eta (0.704, the paper's) in 4 x 4 cells (n = 4 blocks), for
    several chains per cell n_m
    (ell = 1.28 sigma) and chain displacements ell (n_m from eq. nm).  Each
    point is a batch of 32 independent replicas (Philox key (8, r)) advanced
    together, melted by 1000 sweeps; Psi of every replica (Delaunay
    neighbours within 2.5 sigma, every cell certified) is measured every 5
    sweeps (every 25 at eta >= 0.69) and the autocorrelation is averaged over
    the replicas by ecmc_autocorrelation_time.  Each point
    runs until the series are at least 20 tau long (at most --tau-max sweeps);
    tau is given in sweeps and in wall time per replica-sweep.  One JSON line
    per point, then the summary."""
    import torch

    import paper_1409_6948_gb300 as P
    from paper_1409_6948_gb300 import ecmc as E

    torch.cuda.set_device(0)
    # Psi every 5 sweeps in the liquid; every 25 at the paper's density, where
    # tau exceeds 2500 sweeps
    N, eta, cells, seed, R = 4096, args.tau_eta, 4, 8, 32
    every = 5 if eta < 0.69 else 25
    L = W.box_side(N, eta)
    lam0 = (W.ETA_HCP - eta) / (2 * W.ETA_HCP)
    pts = []
    settings = [(1, 1.28), (5, 1.28), (20, 1.28), (0, 0.4), (0, 4.0)]
    for nm, ell in settings:
        nm_used = nm or max(1, int(math.floor(N / (cells * cells) * lam0 / ell + 0.5)))
        descs = [dict(N=N, L=L, sigma=1.0, cells_x=cells, cells_y=cells, ell=ell, n_m=nm_used,
                      seed=seed, replica=r) for r in range(R)]
        g = P.Ecmc.batch(descs)
        g.sweep(1000)
        g.synchronize()
        series = []
        n = 0
        tau = float("inf")
        t_sweep = t_psi = 0.0
        n_bad = 0
        while n < args.tau_max:
            for _ in range(400):
                a = time.perf_counter()
                g.sweep(every)
                g.synchronize()
                b = time.perf_counter()
                psi, _, _, bad = g.hexatic(rs=2.5, per_disk=True)
                series.append(psi)
                t_sweep += b - a
                t_psi += time.perf_counter() - b
                n_bad += bad
            n += 400 * every
            # eq. tau averaged over the replicas (ecmc_autocorrelation_time)
            z = np.array(series)            # [samples, replicas]
            tau_s, _ = E.autocorrelation_time(z, max_lag=z.shape[0] // 4)
            tau = every * tau_s
            if n >= 20 * tau:
                break
        cnt = g.counters()
        pt = {"n_m": nm_used, "ell": ell, "tau_sweeps": tau, "sweeps": n, "replicas": R,
              "mean_abs_psi": float(np.mean(np.abs(series))), "uncertified_cells": n_bad,
              "ms_per_batch_sweep": 1e3 * t_sweep / n,
              "ms_per_psi_measurement": 1e3 * t_psi / (n // every),
              "tau_wall_ms_per_replica": tau * 1e3 * t_sweep / n / R,
              "events_per_replica_sweep": cnt.events / max(cnt.sweeps, 1) / R}
        print(json.dumps(pt), flush=True)
        pts.append(pt)
        g.close()
    # the tuning decision of Figs. 5-6: the setting with the smallest tau in
    # wall time
    fin = [p for p in pts if math.isfinite(p["tau_sweeps"])]
    best = min(fin, key=lambda p: p["tau_wall_ms_per_replica"]) if fin else None
    print(json.dumps({"mode": "tau", "workload": "N=4096 eta=%g cells=4x4, 32 replicas" % eta,
                      "lambda0_eq": lam0, "points": pts, "best_tau_wall": best}))
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload in ("batch", "eos"):
        return run_reference_batch(args)
    w, cells, ell = workload(args)
    import oracle

    L = w.L
    nm = args.nm
    if not args.fixed_params and not args.cells and not args.ell and \
            args.workload in ("large", "huge") or args.paper_params:
        cells, ell, sp_nm = oracle.suggest_parameters(w.N, L, 1.0, 2.0)
        nm = nm or sp_nm
    nm = nm or oracle.default_nm(w.N, L, 1.0, cells, cells, ell)
    x, y = W.square_lattice(w.N, L)
    p = oracle.make_params(w.N, L, 1.0, cells, cells, ell, nm, w.seed)
    melt = melt_sweeps(args)
    oracle.sweeps(p, x, y, 0, melt)
    for s in range(args.warmup):
        oracle.sweeps(p, x, y, melt + s, 1)
    st = oracle.Stats()
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.sweeps(p, x, y, melt + args.warmup + s, 1, stats=st)
    dt = time.perf_counter() - t0
    value = st.events / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name + " cells=%dx%d ell=%g" % (cells, cells, ell), "N": w.N,
                   "eta": w.eta, "cells": cells, "ell": ell, "n_m": nm,
                   "parallelism": "replicas",
                   "start": "square lattice, %d untimed sweeps, then %d warm-up sweeps"
                            % (melt, args.warmup)},
        "sweeps_per_s": args.steps / dt,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d full sweeps after %d untimed melt and %d warm-up "
                                   "sweeps" % (args.steps, melt, args.warmup)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import paper_1409_6948_gb300 as P
    from paper_1409_6948_gb300 import ecmc as E

    w, cells, ell = workload(args)
    L = w.L
    descs = None
    if args.workload in ("batch", "eos"):
        descs = batch_descs(args, rank)
        g = P.Ecmc.batch(descs)
        n_total = sum(d["N"] for d in descs)
        wname = ("%d replicas, N %d..%d (%d disks), eta %.3f..%.3f, paper-strategy cells/ell"
                 % (len(descs), min(d["N"] for d in descs), max(d["N"] for d in descs), n_total,
                    min(d["eta"] for d in descs), max(d["eta"] for d in descs)))
    else:
        use_paper = args.paper_params or (not args.fixed_params and not args.cells and
                                          not args.ell and args.workload in ("large", "huge"))
        if use_paper:
            sp = E.suggest_parameters(w.N, L, 1.0, 2.0)
            cells, ell = sp["cells_x"], sp["ell"]
        g = P.Ecmc(w.N, L, 1.0, cells, cells, ell, w.seed)
        g.set_param(E.PARAM_REPLICA, replica_key(rank))
        if use_paper and not args.nm:
            g.set_param(E.PARAM_N_CHAINS, sp["n_m"])
        n_total = w.N
        wname = w.name + " cells=%dx%d ell=%g" % (cells, cells, ell)
    if args.nm:
        g.set_param(E.PARAM_N_CHAINS, args.nm)
    if args.tpc:
        g.set_param(E.PARAM_LANES_PER_CELL, args.tpc)
    g.set_param(E.PARAM_PRECISION, args.prec)
    if args.fmode >= 0:
        g.set_param(E.PARAM_FRAME_MODE, args.fmode)
    if args.persistent >= 0:
        g.set_param(E.PARAM_PERSISTENT, args.persistent)
    if args.dir == "iso":
        g.set_param(E.PARAM_DIR_MODE, E.DIR_ISOTROPIC)
    # a stream of our own (torch's default stream is the legacy NULL stream,
    # which the library reads as "use your own stream")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    g.set_stream(stream)
    nm = int(g.get_param(E.PARAM_N_CHAINS))
    tpc = int(g.get_param(E.PARAM_LANES_PER_CELL))

    # untimed preparation of the input state: melt the lattice
    g.sweep(melt_sweeps(args))
    # warm-up (graphs captured here)
    g.sweep(args.warmup)
    g.synchronize()
    tuned = None
    if (args.autotune or args.workload in ("large", "huge", "batch", "eos")) and \
            not args.no_autotune and not args.tpc and args.fmode < 0 and args.persistent < 0:
        tuned, _ = g.autotune(trial_sweeps=2)
        tpc = int(g.get_param(E.PARAM_LANES_PER_CELL))
        g.sweep(1)
    saved_xy = g.positions().copy() if descs is not None else None
    saved_t = g.sweep_index()

    # timed region: per-kernel CUDA events inside the library (direct
    # launches), one event pair per step on the same stream, L2 flushed
    # between steps outside the timed pairs
    flush = None if args.no_flush else torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32,
                                                    device=dev)
    g.set_param(E.PARAM_TIMING, 1)
    g.reset_stats()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device()) if local == 0 else None
    if clocks:
        clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for a, b in evs:
        if flush is not None:
            flush.zero_()
        a.record(stream)
        g.sweep(1)
        b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    g.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    c = g.counters()
    kt = g.kernel_times()
    kernels_per_sweep = int(g.get_param(E.PARAM_KERNELS_PER_SWEEP))
    persistent = int(g.get_param(E.PARAM_PERSISTENT))
    g.set_param(E.PARAM_TIMING, 0)
    events = c.events
    sweeps = c.sweeps

    if world > 1:
        ms_max, events_all, sweeps_all = combine_over_ranks(ms, events, sweeps, dev)
    else:
        ms_max, events_all, sweeps_all = ms, float(events), float(sweeps)
    value = events_all / (ms_max * 1e-3)

    # batches: the same sweeps again with every candidate tested in FP64,
    # from the same state; the two forms must give the same pressures
    precision_cmp = None
    if descs is not None:
        p32 = [g.replica_pressure(r)[0] for r in range(len(descs))]
        g.set_param(E.PARAM_PRECISION, 0)
        g.set_positions(saved_xy, t0=saved_t)
        g.reset_stats()
        g.set_param(E.PARAM_TIMING, 1)
        torch.cuda.synchronize()
        for a, b in evs:
            if flush is not None:
                flush.zero_()
            a.record(stream)
            g.sweep(1)
            b.record(stream)
        torch.cuda.synchronize()
        ms64 = sum(a.elapsed_time(b) for a, b in evs)
        c64 = g.counters()
        p64 = [g.replica_pressure(r)[0] for r in range(len(descs))]
        g.set_param(E.PARAM_TIMING, 0)
        g.set_param(E.PARAM_PRECISION, args.prec)
        rel = max(abs(a - b) / abs(b) for a, b in zip(p32, p64))
        precision_cmp = {"fp32_screening_events_per_s": events / (ms * 1e-3),
                         "fp64_candidates_events_per_s": c64.events / (ms64 * 1e-3),
                         "speedup": (events / ms) / (c64.events / ms64),
                         "max_rel_pressure_diff": rel, "same_events": c64.events == events,
                         "per_replica_eta_pressure": [(round(d["eta"], 4), p)
                                                      for d, p in zip(descs, p32)]}

    # end to end through the public API: host (pinned) positions in, one
    # sweep, positions out, every step
    e2e = None
    if not args.skip_e2e:
        host = torch.empty(2 * n_total, dtype=torch.float64, pin_memory=True)
        g.positions(host.numpy())
        t_idx = g.sweep_index()
        g.reset_stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(args.steps):
            g.set_positions(host.numpy(), t0=t_idx + s)
            g.sweep(1)
            g.positions(host.numpy())
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ce = g.counters()
        e2e = {"value": ce.events / dt, "unit": UNIT, "h2d_bytes_per_step": 16 * n_total,
               "d2h_bytes_per_step": 16 * n_total, "timer": "host wall clock"}

    line = None
    if rank == 0:
        phase_avg_ms = kt.phase_ms / max(kt.phase_launches, 1)
        iters = c.events + c.wall_hits + c.chains
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
        smem_peak, fp64_probe = P.ecmc.device_peaks()
        # the configuration the ncu counters were taken in
        fm_used = int(g.get_param(E.PARAM_FRAME_MODE))
        captured = (fm_used if (persistent and tpc == 8 and descs is None and args.dir == "axis"
                                and args.prec == 1 and fm_used in FUSED_CAPTURES) else None)
        cpu = None
        if not args.skip_cpu and descs is None:
            cpu = cpu_baseline(w, cells, ell, nm, args.cpu_seconds, melt_sweeps(args),
                               dir_mode=2 if args.dir == "iso" else 0)
        elif not args.skip_cpu:
            cpu = cpu_baseline_batch(descs, args.cpu_seconds)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "N": n_total, "eta": w.eta if descs is None else None,
                       "cells": cells if descs is None else None,
                       "ell": ell if descs is None else None,
                       "n_m": nm if descs is None else None, "lanes_per_cell": tpc,
                       "autotuned": tuned,
                       "screening": "fp32" if args.prec else "fp64",
                       "l2": "none" if args.no_flush else "flushed (256 MB write) between steps",
                       "start": "square lattice, %d untimed sweeps, then %d warm-up sweeps"
                                % (melt_sweeps(args), args.warmup),
                       "parallelism": "replicas x%d" % world,
                       "launch": "persistent sweep kernel" if persistent else "per-phase kernels",
                       "directions": "isotropic" if args.dir == "iso" else "alternating axes"},
            "sweeps_per_s": sweeps_all / (ms_max * 1e-3),
            "events_per_sweep": events / max(sweeps, 1),
            "per_sweep": {"chains": c.chains / max(sweeps, 1),
                          "frozen_hits": c.frozen_hits / max(sweeps, 1),
                          "wall_hits": c.wall_hits / max(sweeps, 1),
                          "fp64_evals": c.fp64_evals / max(sweeps, 1)},
            "kernel_ms_per_sweep": {"bin": kt.bin_ms / max(sweeps, 1),
                                    "frame": kt.frame_ms / max(sweeps, 1),
                                    "chain": kt.phase_ms / max(sweeps, 1),
                                    "reduce": kt.other_ms / max(sweeps, 1)},
            "roofline": chain_roofline(w, descs, c, iters, kt, args.prec, smem_peak, persistent,
                                       captured),
            "fp64_pipe": fp64_pipe(iters, kt, n_sm, sm_mhz, fp64_probe, persistent, captured),
            "latency": latency_ceiling(g, descs, cells, c, kt, clk, sm_mhz),
            # per sweep: draws, binning, the persistent sweep kernel (or 4 x frame
            # builder + chain kernel), chunk sums, end of sweep
            "gpu_launches": kernels_per_sweep * args.steps * world,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        if precision_cmp is not None:
            line["precision_comparison"] = precision_cmp
        print(json.dumps(line))
    g.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def smem_bytes_per_event(w, c, iters, prec):
    """ALGORITHMIC shared-memory bytes per collision event: an event must
    inspect the disks whose centres lie in the strip that can hold the first
    hit, area 2 sigma (sigma + lambda0) with lambda0 the measured mean free
    path, at 8 B (FP32 x, y) or 16 B (FP64) each, plus 16 B to read and write
    the mover.  Returns (bytes, disks, lambda0)."""
    rho = w.N / (w.L * w.L)
    lam0 = c.sum_disp / iters
    disks = rho * 2.0 * (1.0 + lam0)
    return disks * (8.0 if prec else 16.0) + 16.0, disks, lam0


def chain_roofline(w, descs, c, iters, kt, prec, smem_peak, persistent, captured):
    """The dominant kernel against shared-memory bandwidth: algorithmic bytes
    per event x events per launch / the kernel's average launch time (CUDA
    events on the launching stream) / the measured ld.shared.v4 peak.  traffic:
    DRAM read + write per launch from the ncu capture, scaled to this workload
    by the disks, when the kernel runs in the captured configuration."""
    launches = max(kt.phase_launches, 1)
    if descs is not None or iters <= 0 or kt.phase_launches <= 0:
        return None
    per, disks, lam0 = smem_bytes_per_event(w, c, iters, prec)
    launch_ms = kt.phase_ms / launches
    events_per_launch = c.events / launches
    achieved = per * events_per_launch / (launch_ms * 1e-3) / 1e9
    cap = fused_capture(captured)
    traffic = (cap["dram_bytes"] * w.N / FUSED_CAPTURE_N) if cap else None
    return {"kernel": "k_sweep_fused (persistent sweep kernel)" if persistent
                      else "k_phase (chain kernel)",
            "bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
            "frac": achieved / smem_peak if smem_peak else None, "traffic": traffic,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch "
                               "at N=%d, scaled by the disks" % FUSED_CAPTURE_N)
                              if cap else None,
            "bytes_per_event": per, "candidates_per_event": disks, "mean_free_path": lam0,
            "events_per_launch": events_per_launch, "launch_ms": launch_ms,
            "peak_source": "ld.shared.v4 probe on this device in this run (no shared-memory "
                           "figure in MEASURED_PEAKS.json)"}


def fp64_pipe(iters, kt, n_sm, sm_mhz, fp64_probe_gflops, persistent, captured):
    """Use of the FP64 pipe by the dominant kernel, in warp-instructions: FP64
    warp-instructions per launch (per iteration from the ncu capture, times
    this run's iterations) x SM cycles one FP64 warp-instruction occupies
    (from the FMA probe: SMs x clock / (FMA/s / 32 lanes)) / SM cycles of the
    launch (SMs x clock x average launch time)."""
    cap = fused_capture(captured)
    if not (persistent and cap) or kt.phase_launches <= 0 or not fp64_probe_gflops:
        return None
    launch_s = kt.phase_ms / kt.phase_launches * 1e-3
    winst = cap["fp64_winst"] / FUSED_ITERATIONS_CAPTURE * iters / kt.phase_launches
    clk = sm_mhz * 1e6
    cyc_per_winst = n_sm * clk / (fp64_probe_gflops * 1e9 / 2.0 / 32.0)
    sm_cycles = n_sm * clk * launch_s
    return {"warp_instructions_per_launch": winst,
            "warp_instructions_per_iteration": cap["fp64_winst"] / FUSED_ITERATIONS_CAPTURE,
            "cycles_per_warp_instruction": cyc_per_winst, "sm_cycles_per_launch": sm_cycles,
            "frac": winst * cyc_per_winst / sm_cycles,
            "ncu_pipe_active_pct_at_capture": cap["fp64_pipe_pct"],
            "probe_fp64_gflops": fp64_probe_gflops,
            "source": "FP64 warp-instructions per iteration from ncu at N=%d" % FUSED_CAPTURE_N}


def latency_ceiling(g, descs, cells, c, kt, clk, sm_mhz):
    """Cycles one event costs a chain, from the dominant launch's time, the
    SM clock and the chains the launch runs at once; and the events/s that
    rate would give if every cell of a colour phase ran at the same time."""
    from paper_1409_6948_gb300 import ecmc as E

    flight = g.get_param(E.PARAM_CHAINS_IN_FLIGHT)
    if descs is not None or flight <= 0 or kt.phase_launches <= 0 or c.events <= 0:
        return None
    mhz = (clk or {}).get("sm_mhz") or sm_mhz
    launch_ms = kt.phase_ms / kt.phase_launches
    events_per_launch = c.events / kt.phase_launches
    cyc = launch_ms * 1e-3 * mhz * 1e6 * flight / events_per_launch
    active = cells * cells / 4
    return {"chains_in_flight": flight, "active_cells_per_phase": active,
            "cycles_per_event_per_chain": cyc, "sm_mhz": mhz,
            "ceiling_all_active_cells": active * mhz * 1e6 / cyc, "unit": "events/s"}


def run_reference_batch(args):
    """The oracle as the reference arm on a replica batch: each step is one
    sweep of one replica, the replicas taken in turn."""
    import oracle

    descs = batch_descs(args, 0, reference=True)
    states = []
    for d in descs:
        x, y = W.square_lattice(d["N"], d["L"])
        p = oracle.make_params(d["N"], d["L"], 1.0, d["cells_x"], d["cells_y"], d["ell"],
                               d["n_m"], d["seed"], d["replica"])
        states.append([p, x, y, 0])
    for i in range(args.warmup):
        s = states[i % len(states)]
        oracle.sweeps(s[0], s[1], s[2], s[3], 1)
        s[3] += 1
    st = oracle.Stats()
    t0 = time.perf_counter()
    for i in range(args.steps):
        s = states[(args.warmup + i) % len(states)]
        oracle.sweeps(s[0], s[1], s[2], s[3], 1, stats=st)
        s[3] += 1
    dt = time.perf_counter() - t0
    value = st.events / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "replicas": len(descs)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d single-replica sweeps, replicas in turn" % args.steps},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.grid:
        return run_grid(args)
    if args.listbias:
        return run_listbias(args)
    if args.fig3:
        return run_fig3(args)
    if args.stripes:
        return run_stripes(args)
    if args.dim3:
        return run_dim3(args)
    if args.tau:
        return run_tau(args)
    if args.gr:
        return run_gr(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

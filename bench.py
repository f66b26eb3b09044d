#!/usr/bin/env python
"""Throughput benchmark of the LELBM time step on GB300 (one JSON line on rank 0).

Default workload: the seeded 2D four-quadrant Riemann problem at 4096 x 4096 cells with
the learned EPR warm start, on the mixed path (FP32 Newton, double-float correction and
streaming judged at the FP64 tolerance), compared with the plain FP64 path (Eq. IID13
start) from the same state: MLUPS of both and the L1 density difference between them.
The FP32 path is reported beside them with its own L1.  A step is one time step of every
cell (fluid-boundary fill, collision, LAS, EPR, moment streaming).  MLUPS = interior cell
updates per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batch1d|hotbox2d|riemann2d|cylinder2d|hotbox3d|riemann3d]

--impl reference times the plain FP64 CPU oracle (the correctness reference) on a
bounded sample of the same workload.  Under torchrun each rank runs its own batch
(weak scaling, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline, FP32+learned-EPR vs plain FP64, at matched L1 error"

# Algorithmic FP64 work per stencil point and Newton pass: exponent (N FMA), residual (N FMA)
# and the packed Jacobian (N(N+1)/2 FMA) for N constraints; moment streaming: one multiply and
# one add per stored moment.  Exponentials are not counted.
N_F = {1: 4, 2: 10, 3: 19}
N_G = {1: 3, 2: 6, 3: 10}
N_M = {1: 6, 2: 11, 3: 17}


# DRAM bytes (read + write) per time step of the timed kernel, from one ncu capture of the
# same kernel on the same workload and launch of one step (the summaries in profiles/).
# Configurations without a capture report traffic null.  An entry whose kernel has changed
# since its capture is kept under STALE_DRAM_PER_STEP: the line reports traffic null and
# gives the old figure, labelled, beside it.
DRAM_PER_STEP = {}
STALE_DRAM_PER_STEP = {
    # captured while the mixed cell update stepped its block as one group of twelve warps; it
    # now steps two groups of six warps with their own barriers (same memory accesses)
    ("riemann2d", 1024, "mixed", "learned"): (999.0e6, "profiles/cell_update_mixed_riemann2d_1024.md"),
    ("riemann2d", 4096, "mixed", "learned"): (16.61e9, "profiles/cell_update_mixed_riemann2d_1024.md (4096^2 capture)"),
}


def newton_flops(n: int) -> int:
    return 2 * (2 * n + n * (n + 1) // 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="riemann2d",
                    choices=["batch1d", "hotbox2d", "riemann2d", "cylinder2d", "hotbox3d", "riemann3d"])
    ap.add_argument("--n-batch", type=int, default=4096)
    ap.add_argument("--n", type=int, default=None, help="grid size (default 4096 in 2D, 128 in 3D)")
    ap.add_argument("--rt", type=float, default=0.5, help="hot-box temperature")
    ap.add_argument("--precision", default="mixed", choices=["fp32", "mixed", "fp64"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-path comparison run")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default persistent launch shape")
    ap.add_argument("--warmstart", default="learned", choices=["learned", "maxwell", "stored"],
                    help="EPR Newton start of the timed path: the trained MLP or Eq. (IID13)")
    ap.add_argument("--mlp-gate", type=float, default=1e-3,
                    help="timed path: learned start only for cells whose constraints depart from equilibrium "
                         "by at least this much (0: every cell); the FP64 comparison runs use the network everywhere")
    ap.add_argument("--full-run", action="store_true",
                    help="run the workload's whole configured step count on the timed path and on the "
                         "plain FP64 path from the same state; report both MLUPS and the final L1 density "
                         "difference (one JSON line, metric: L1 after the full run)")
    ap.add_argument("--deterministic", action="store_true",
                    help="FP64 2D path: moment streaming as a fixed-order gather (no atomics)")
    ap.add_argument("--per-step", action="store_true", help="1D batch: one launch per step instead of the "
                    "persistent batch kernel")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    a = ap.parse_args()
    if a.n is None:
        a.n = 128 if a.workload.endswith("3d") else 4096
    if a.workload.endswith("3d"):  # the 3D step is the FP64 path from Eq. (IID13)
        a.precision, a.warmstart, a.no_compare = "fp64", "maxwell", True
    return a


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ---------------------------------------------------------------------------
def rank_reduce(x: float, op: str, world: int, device) -> float:
    """x combined over the ranks of the job: "max" (the slowest rank's time) or "sum" (the
    work of all ranks); x itself when the job has one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_mlups(units_all_ranks: float, steps: int, ms_slowest: float) -> float:
    """Cell updates of all ranks per second of the slowest rank, in millions."""
    return units_all_ranks * steps / (ms_slowest / 1e3) / 1e6


def make_workload(args, rank):
    from paper_2508_06911_gb300 import workloads as W

    if args.workload == "batch1d":
        w = W.riemann_1d_batch(n_batch=args.n_batch, seed_index=1 + 1000 * rank)
        desc = {"workload": f"riemann1d_batch_{args.n_batch}", "dims": 1, "instances": args.n_batch,
                "lengths": "256-4096 log-uniform", "pressure_ratio": "10-1000", "mach_max": 3,
                "interior_cells": int(w.lengths.sum()), "pad_cells": int(2 * w.pads.sum())}
        return w, desc
    if args.workload == "hotbox2d":
        w = W.hot_box(2, args.n, args.rt)
        return w, {"workload": f"hotbox2d_{args.n}x{args.n}_RT{args.rt}", "dims": 2, "u": [10, 10],
                   "interior_cells": args.n * args.n}
    if args.workload == "cylinder2d":
        # Mach-3 slip-wall cylinder, 2n x n cells, diameter n/8 (2048 x 1024, D = 128 at n = 1024)
        w = W.cylinder_2d(nx=2 * args.n, ny=args.n, diameter=args.n // 8)
        fluid = int((w.solid == 0).sum())
        return w, {"workload": w.name, "dims": 2, "interior_cells": fluid, "solid_cells": int(w.solid.sum()),
                   "mach": 3.0, "boundary": "inflow x-, outflow elsewhere, slip-wall cylinder"}
    if args.workload == "hotbox3d":
        w = W.hot_box_3d(args.n, args.rt)
        return w, {"workload": f"hotbox3d_{args.n}^3_RT{args.rt}", "dims": 3, "u": [10, 10, 10],
                   "interior_cells": args.n ** 3}
    if args.workload == "riemann3d":
        w = W.riemann_3d(n=args.n, seed_index=6 + 1000 * rank)
        return w, {"workload": f"riemann3d_{args.n}^3", "dims": 3, "interior_cells": args.n ** 3,
                   "octants": "rho U[0.1,1.5], |u| <= 1.5, p U[0.03,1.5], RT_max/RT_min <= 8"}
    w = W.riemann_2d(n=args.n, seed_index=2 + 1000 * rank)
    return w, {"workload": f"riemann2d_{args.n}x{args.n}", "dims": 2, "interior_cells": args.n * args.n}


def clock_sampler_start():
    out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=out, stderr=subprocess.DEVNULL)
    except Exception:
        p = None
    return p, out.name


def clock_sampler_stop(state, gpu_index=0):
    p, path = state
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or not f[0].isdigit() or int(f[0]) != gpu_index:
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    os.unlink(path)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def small_2d(args, n):
    """An n x n (cylinder: 2n x n; 3D: 8^3) instance of the workload for the CPU oracle."""
    from paper_2508_06911_gb300 import workloads as W

    if args.workload == "hotbox3d":
        return W.hot_box_3d(8, args.rt), 8 ** 3
    if args.workload == "riemann3d":  # the same octant states on a periodic 8^3 box (no pad cells)
        return W.riemann_3d(n=8, periodic=True), 8 ** 3
    if args.workload == "hotbox2d":
        return W.hot_box(2, n, args.rt), n * n
    if args.workload == "cylinder2d":
        w = W.cylinder_2d(nx=2 * n, ny=n, diameter=max(n // 8, 2))
        return w, int((w.solid == 0).sum())
    return W.riemann_2d(n=n, seed_index=2), n * n


# The oracle on the host cores: one process per core (spawned, so that no CUDA state is
# inherited), each running the unchanged serial oracle on whole instances.
_POOL_W = None


def _pool_init(workload, n_batch, n2d, rt):
    global _POOL_W
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle as O
    from paper_2508_06911_gb300 import workloads as W

    O.lib()
    if workload == "batch1d":
        _POOL_W = W.riemann_1d_batch(n_batch=n_batch, seed_index=1)
    else:
        ns = argparse.Namespace(workload=workload, rt=rt)
        _POOL_W = small_2d(ns, n2d)


def _pool_task(b):
    """One time step of instance b (1D) or of the small 2D instance; returns interior cells."""
    from parity_util import oracle_1d_instance, oracle_2d, oracle_3d

    if isinstance(_POOL_W, tuple):
        (oracle_3d if _POOL_W[0].__class__.__name__ == "Grid3D" else oracle_2d)(_POOL_W[0], 1)
        return _POOL_W[1]
    oracle_1d_instance(_POOL_W, b, 1)
    return int(_POOL_W.lengths[b])


def oracle_pool(args, n2d):
    import concurrent.futures as cf
    import multiprocessing as mp

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    ex = cf.ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn"), initializer=_pool_init,
                                initargs=(args.workload, args.n_batch, n2d, args.rt))
    list(ex.map(_pool_task, range(cores)))  # start every worker before any timing
    return ex, cores


def cpu_baseline(args, budget_s=10.0):
    """The CPU oracle, as it stands (serial FP64 C), on every host core, on a bounded
    sample of the workload: whole instances (1D) or steps of a small instance (2D)."""
    import concurrent.futures as cf

    ex, cores = oracle_pool(args, 64)
    n_units = args.n_batch if args.workload == "batch1d" else None
    t0 = time.perf_counter()
    cells, k, pending = 0, 0, set()
    while True:
        while (len(pending) < 2 * cores and time.perf_counter() - t0 < budget_s
               and (n_units is None or k < n_units)):
            pending.add(ex.submit(_pool_task, k))
            k += 1
        if not pending:
            break
        done, pending = cf.wait(pending, return_when=cf.FIRST_COMPLETED)
        cells += sum(f.result() for f in done)
    dt = time.perf_counter() - t0
    ex.shutdown()
    unit = "instances of the batch" if args.workload == "batch1d" else "steps of a 64-cell-wide instance"
    return {"value": cells / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{k} {unit} ({cells} interior cell updates), one process per core",
            "seconds": round(dt, 2)}


# ---------------------------------------------------------------------------
def run_reference(args):
    """Reference arm: the CPU oracle, each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, desc = make_workload(args, 0)
    ex, cores = oracle_pool(args, 48)
    per_step = []
    cells_step = 0

    per = 4 * cores

    def one_step():
        # one step: the first 4 x cores instances (1D) or 4 x cores steps of the small instance
        nonlocal cells_step
        c = sum(ex.map(_pool_task, range(per)))
        cells_step = c
        return c

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    tot = 0
    for _ in range(args.steps):
        ts = time.perf_counter()
        tot += one_step()
        per_step.append(time.perf_counter() - ts)
    dt = time.perf_counter() - t0
    ex.shutdown()
    v = tot / dt / 1e6
    sample = (f"first {per} instances of the batch ({cells_step} interior cells) per step, one process per core"
              if args.workload == "batch1d" else
              f"{per} steps of a small instance of the workload ({cells_step} cell updates) per step")
    line = {"metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": desc, "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2508_06911_gb300 import build as B, lelbm as L
    from paper_2508_06911_gb300.solver import Solver

    B.build()
    # FMA throughput of this GPU's FP32 and FP64 pipes (the ALU-roofline denominators)
    fp32_peak = L.lelbm_fma_peak(False)
    fp64_peak = L.lelbm_fma_peak(True)
    w, desc = make_workload(args, rank)
    # a dedicated stream: the legacy default stream has handle 0, which the ABI reads as
    # "create a stream of your own"
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    D = desc["dims"]
    interior = desc["interior_cells"]
    prec = {"fp32": L.LELBM_FP32, "mixed": L.LELBM_MIXED, "fp64": L.LELBM_FP64}

    weights = None
    # the four-quadrant workload uses the network trained along the 2000-step 1024^2 run (the same
    # generator at 1024^2), the others the network trained on diverse 2D states
    wname = "warmstart_2d_quadrants.npy" if args.workload == "riemann2d" else f"warmstart_{D}d.npy"
    wpath = os.path.join(ROOT, "paper_2508_06911_gb300", "weights", wname)
    if D < 3 and (args.warmstart == "learned" or not args.no_compare):
        if os.path.exists(wpath):
            weights = np.load(wpath)
        else:  # no trained network shipped: train one on pairs recorded by the plain solver
            from paper_2508_06911_gb300 import warmstart as WS
            from paper_2508_06911_gb300 import workloads as W
            src = (Solver.riemann1d(W.riemann_1d_batch(n_batch=1024, seed_index=11)) if D == 1
                   else Solver.grid2d(W.riemann_2d(n=512, seed_index=12)))
            X, Y = WS.record_pairs(src, steps=2)
            weights, _ = WS.train(D, X, Y)
            src.close()

    def make(precision, start):
        kw = dict(stream=stream.cuda_stream, precision=prec[precision])
        if args.deterministic and precision == "fp64":
            kw["deterministic"] = 1
        s_ = Solver.riemann1d(w, **kw) if D == 1 else (Solver.grid2d(w, **kw) if D == 2 else Solver.grid3d(w, **kw))
        if start == "learned" and weights is not None:
            L.lelbm_set_mlp(s_.h, weights)
            if precision == args.precision and precision != "fp64":
                L.lelbm_set_mlp_gate(s_.h, args.mlp_gate)
        if start == "stored":
            s_.set_warmstart(True)
        return s_

    persistent = D == 1 and not args.per_step

    def advance(s, n):
        if persistent:
            s.run_batch(n)
        else:
            s.step(n)

    def timed(s, sample_clocks):
        if persistent and not args.no_autotune:
            s.autotune(1)
        advance(s, args.warmup)
        torch.cuda.synchronize()
        L.lelbm_reset_stats(s.h)
        L.lelbm_set_timing(s.h, True)
        barrier()
        torch.cuda.synchronize()
        clk = clock_sampler_start() if sample_clocks else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        advance(s, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = clock_sampler_stop(clk, local) if sample_clocks else None
        ms = rank_reduce(e0.elapsed_time(e1), "max", world, "cuda")
        return ms, s.stats(), s.synchronize(), clocks

    s = make(args.precision, args.warmstart)
    state_bytes = s.n_mom * s.n_cells * 8
    ms, st, status, clocks = timed(s, True)
    units = rank_reduce(interior, "sum", world, "cuda")  # each rank has its own seeded batch
    value = whole_job_mlups(units, args.steps, ms)

    def summary(ms_, st_):
        h_ = list(st_.newton_hist)
        return {"value": whole_job_mlups(units, args.steps, ms_), "ms_per_step": ms_ / args.steps,
                "points_fp32": st_.points_32, "points_fp64_newton": st_.points_f + st_.points_g,
                "newton_mean_updates": sum(i * x for i, x in enumerate(h_)) / max(sum(h_), 1),
                "start_retry": st_.mlp_retry}

    compare = None
    warm_starts = None
    fp32_path = None
    if not args.no_compare:
        other = "fp64" if args.precision != "fp64" else "fp32"
        s2 = make(other, "maxwell")  # the plain path: Eq. (IID13) start
        ms2, st2, _, _ = timed(s2, False)
        r1 = s.get_moments()[0]
        r2 = s2.get_moments()[0]
        l1 = float(np.abs(r1 - r2).sum() / np.abs(r2 if other == "fp64" else r1).sum())
        compare = {"precision": other, **summary(ms2, st2),
                   "kernel_ms": st2.cell_kernel_ms / max(st2.cell_kernel_launches, 1),
                   "l1_density_rel": l1, "warmstart": "maxwell",
                   "note": "both runs from the same state, warmup + steps each"}
        s2.close()
        # every warm start on the timed precision, and the stored and learned ones on the other
        warm_starts = {args.warmstart: summary(ms, st)}
        for start in ("maxwell", "stored", "learned"):
            if start == args.warmstart or (start == "learned" and weights is None):
                continue
            s3 = make(args.precision, start)
            ms3, st3, _, _ = timed(s3, False)
            warm_starts[start] = summary(ms3, st3)
            s3.close()
        for start in ("stored", "learned"):
            if start == "learned" and weights is None:
                continue
            s4 = make(other, start)
            ms4, st4, _, _ = timed(s4, False)
            compare[start] = summary(ms4, st4)
            s4.close()
        if args.precision == "mixed":
            # the FP32 path (FP32 Newton to 3e-4, FP32 streaming) from the same state and start
            s5 = make("fp32", args.warmstart)
            ms5, st5, _, _ = timed(s5, False)
            r5 = s5.get_moments()[0]
            fp32_path = {**summary(ms5, st5), "warmstart": args.warmstart,
                         "l1_density_rel": float(np.abs(r5 - r2).sum() / np.abs(r2).sum()),
                         "note": "L1 against the FP64 path after the same steps"}
            s5.close()

    # dominant kernel: the fused cell update, bound by its ALU pipe: FP64 on the FP64 path,
    # FP32 on the FP32 and mixed paths (the mixed path's double-float passes run on the FP32
    # pipe).  Algorithmic work (the naive assembly): per stencil point and Newton pass
    # of a population 2(2N + N(N+1)/2) FLOP (exponent, residual, packed Jacobian), per
    # streamed point 2 n_mom FLOP; a double-float correction pass counts as a Newton pass,
    # a double-float streaming pass as streaming.  One timed launch covers args.steps steps
    # on the persistent path.
    launches = max(st.cell_kernel_launches, 1)
    kern_ms = st.cell_kernel_ms / launches
    both = newton_flops(N_F[D]) + (newton_flops(N_G[D]) if w.K > 0 else 0)
    flops64 = (st.points_f * newton_flops(N_F[D]) + st.points_g * newton_flops(N_G[D])) / launches
    flops32 = st.points_32 * both / launches
    flops32 += st.points_df_corr * (both / (2 if w.K > 0 else 1)) / launches
    flops_ms = st.points_ms * 2 * N_M[D] / launches
    if args.precision == "fp64":
        flops64 += flops_ms
    else:
        flops32 += flops_ms
    steps_per_launch = args.steps if persistent else 1
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    alg_bytes = (2 * s.n_mom * 8 + 1) * interior * steps_per_launch  # read state + write next + type byte
    prec_id = {"fp64": 0, "mixed": 1, "fp32": 2}[args.precision]
    sec = kern_ms / 1e3
    probe = "lelbm_fma_peak: FMA probe kernel run by this benchmark on this GPU"
    if args.precision != "fp64":
        main_side = {"achieved": flops32 / sec / 1e12, "peak": fp32_peak / 1e12, "peak_source": probe + " (FP32)"}
        other_side = {"fp64_side": {"achieved_tflops": flops64 / sec / 1e12, "peak_tflops": fp64_peak / 1e12,
                                    "note": "FP64 EPR of the cells the FP32 or double-float finish leaves"}}
    else:
        main_side = {"achieved": flops64 / sec / 1e12, "peak": fp64_peak / 1e12, "peak_source": probe + " (FP64)"}
        other_side = {"fp32_side": {"achieved_tflops": flops32 / sec / 1e12, "peak_tflops": fp32_peak / 1e12}}
    size = args.n_batch if args.workload == "batch1d" else args.n
    dram = DRAM_PER_STEP.get((args.workload, size, args.precision, args.warmstart))
    stale = None if dram else STALE_DRAM_PER_STEP.get((args.workload, size, args.precision, args.warmstart))
    roofline = {"bound": "alu", "achieved": main_side["achieved"], "peak": main_side["peak"], "unit": "TFLOP/s",
                "frac": main_side["achieved"] / main_side["peak"],
                "traffic": dram[0] * steps_per_launch if dram else None,
                "traffic_source": (f"{dram[1]}: ncu dram bytes of one step x {steps_per_launch} steps per launch"
                                   if dram else None),
                **({"traffic_stale": {"value": stale[0] * steps_per_launch,
                                      "source": f"{stale[1]}, captured before the kernel's last change"}}
                   if stale else {}),
                "peak_source": main_side["peak_source"],
                "kernel": (f"batch_persistent_kernel<{prec_id}>" if persistent else
                           ("cell3d_kernel" if D == 3 else f"cell_update_kernel<{D},{prec_id}>")
                           + (" + gather2d_kernel" if args.deterministic and args.precision == "fp64" else "")),
                "kernel_ms": kern_ms, "steps_per_launch": steps_per_launch, **other_side,
                "hbm": {"achieved_gbs": alg_bytes / sec / 1e9, "peak_gbs": hbm_peak,
                        "frac": alg_bytes / sec / 1e9 / hbm_peak,
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"}}
    # per step: pad fill (padded grids), the warm-start network (learned start), the cell update,
    # the gather (deterministic streaming)
    launches_per_step = (1 + (s.n_cells > interior) + (args.warmstart == "learned" and weights is not None)
                         + (args.deterministic and args.precision == "fp64"))
    hist = list(st.newton_hist)
    solves = sum(hist)
    mean_updates = sum(i * h for i, h in enumerate(hist)) / max(solves, 1)

    e2e = None
    if not args.no_e2e:
        host = torch.empty((s.n_mom, s.n_cells), dtype=torch.float64, pin_memory=True).numpy()
        s.get_moments()
        L.lelbm_get_moments(s.h, host)
        ke = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            L.lelbm_set_moments(s.h, host)
            advance(s, 1)
            L.lelbm_get_moments(s.h, host)
        dt = rank_reduce(time.perf_counter() - t0, "max", world, "cuda")
        e2e = {"value": whole_job_mlups(units, ke, dt * 1e3), "unit": "MLUPS", "h2d_bytes_per_step": state_bytes,
               "d2h_bytes_per_step": state_bytes, "steps": ke}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args)

    if rank == 0:
        if args.deterministic and args.precision == "fp64":
            desc["streaming"] = "deterministic gather"
        desc.update({"precision": args.precision, "l2": f"inputs larger than L2 (state {state_bytes / 1e6:.0f} MB x 2 buffers)"
                     if 2 * state_bytes > 129e6 else "state fits in L2",
                     "parallelism": f"{world} independent replica(s)" if world > 1 else "single GPU"})
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32+f64",
                "data": "synthetic (seeded)",
                "config": desc, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "compare": compare,
                "speedup_vs_fp64": (value / compare["value"]) if (compare and args.precision != "fp64") else None,
                "warmstart": args.warmstart if (args.warmstart != "learned" or weights is not None) else "maxwell",
                "mlp_gate": args.mlp_gate if (args.warmstart == "learned" and weights is not None) else None,
                "warm_starts": warm_starts, "fp32_path": fp32_path, "points_fp32": st.points_32,
                "points_df_corr": st.points_df_corr, "points_df_stream": st.points_df,
                "fma_peaks_tflops": {"fp32": fp32_peak / 1e12, "fp64": fp64_peak / 1e12},
                "points_fp64_newton": st.points_f + st.points_g, "mlp_retry": st.mlp_retry,
                "mlp_cells_frac": st.mlp_cells / max(st.cells, 1),
                "gpu_launches": 1 if persistent else int(args.steps * launches_per_step),
                "clocks": clocks, "status": L.STATUS.get(status, status),
                "newton_mean_updates": mean_updates, "fallback_eq": st.fallback_eq,
                "fallback_mx": st.fallback_mx, "judge_redo": st.judge_redo, "q_max": st.q_max,
                "disp_max": st.disp_max}
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def run_full(args):
    """The workload's whole run (its configured step count) on the timed path and on the plain
    FP64 path (Eq. IID13 start) from the same initial state: MLUPS of each and the relative L1
    density difference between the two final states (the accuracy half of the metric)."""
    import torch

    from paper_2508_06911_gb300 import build as B, lelbm as L
    from paper_2508_06911_gb300.solver import Solver

    torch.cuda.set_device(0)
    B.build()
    w, desc = make_workload(args, 0)
    D = desc["dims"]
    if D != 2:
        raise SystemExit("--full-run covers the 2D workloads")
    nsteps = int(w.steps)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = {"fp32": L.LELBM_FP32, "mixed": L.LELBM_MIXED, "fp64": L.LELBM_FP64}
    wname = "warmstart_2d_quadrants.npy" if args.workload == "riemann2d" else f"warmstart_{D}d.npy"
    wpath = os.path.join(ROOT, "paper_2508_06911_gb300", "weights", wname)
    res = {}
    rho = {}
    for name, precision, start in (("timed", args.precision, args.warmstart), ("fp64", "fp64", "maxwell")):
        kw = dict(stream=stream.cuda_stream, precision=prec[precision])
        s = Solver.grid2d(w, **kw)
        if start == "learned" and os.path.exists(wpath):
            L.lelbm_set_mlp(s.h, np.load(wpath))
            if precision != "fp64":
                L.lelbm_set_mlp_gate(s.h, args.mlp_gate)
        if start == "stored":
            s.set_warmstart(True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        while done < nsteps:  # in chunks, so that a very long run is not one enqueue
            k = min(500, nsteps - done)
            s.step(k)
            done += k
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = s.stats()
        res[name] = {"precision": precision, "warmstart": start, "steps": nsteps, "seconds": ms / 1e3,
                     "value": desc["interior_cells"] * nsteps / (ms / 1e3) / 1e6, "status": L.STATUS.get(s.synchronize()),
                     "fallback_mx": st.fallback_mx, "judge_redo": st.judge_redo}
        rho[name] = s.get_moments()[0]
        s.close()
    l1 = float(np.abs(rho["timed"] - rho["fp64"]).sum() / np.abs(rho["fp64"]).sum())
    desc.update({"precision": args.precision, "steps": nsteps})
    print(json.dumps({"metric": "relative L1 density difference from the plain FP64 path after the full run",
                      "value": l1, "unit": "relative", "n_gpus": 1, "higher_is_better": False,
                      "data": "synthetic (seeded)", "config": desc, "runs": res,
                      "speedup_vs_fp64": res["timed"]["value"] / res["fp64"]["value"]}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.full_run:
        run_full(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the full multigrid solve for -Laplace(u) + u^3 = g (Algorithm 3.2).

Workload: 2D unit square, P1 on the right-triangle mesh, coarse H = 1/8, 8 uniform
refinements (2049 x 2049 nodes, 4,190,209 fine DOFs), u* = 8 seeded sin modes
(k, l in 1..6, N(0,1) amplitudes; seed = rank), m = 2 V(2,2) cycles, p = 1.

One step = one fmg_solve of that problem (level-1 Newton, every level's prolongation,
linearized right-hand side, V-cycles, augmented-space Newton and update) with the inputs
resident in HBM.  `value` is fine DOFs/s of the mixed-precision path (FP32 cycles inside
FP64 defect correction); the FP64 path is timed beside it ("fp64").  L2 is flushed
between steps (a 512 MB write outside the timed events).

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
Under torchrun each rank solves its own instance (independent problems, weak scaling);
the reported time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMG fine DOFs/s to discretization error, mixed vs FP64; HBM GB/s; p50/p99"
FP64_FLOPS_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9  # SMs x DFMA/clk x 2 flop x max SM clock
WORKLOAD = "2D unit square P1, H=1/8, 8 refinements (2049x2049 nodes, 4,190,209 fine DOFs), u^3, 8 sin modes"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--refinements", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            hbm = d.get("hbm_gbs") or d.get("hbm_GBps")
            if hbm:
                return float(hbm), "of measured"
        except Exception:
            pass
    return 6800.0, "of fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(torch):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        return dist, world, rank, local
    return None, 1, 0, local


def barrier(dist, torch):
    if dist is not None:
        if torch.cuda.is_available():
            dist.barrier(device_ids=[torch.cuda.current_device()])
        else:
            dist.barrier()


def max_over_ranks(dist, torch, x: float) -> float:
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------- CPU oracle

def oracle_sample(refinements: int, repeats: int, seed: int = 0):
    """FP64 oracle FMG on a bounded sample of the workload: same H, fewer refinements."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:  # pragma: no cover
        threadpool_limits = None
    from oracle import fmg_oracle as O
    from paper_1611_05677_gb300 import workloads as W

    prob = W.config_large_2d(seed=seed, refinements=refinements)
    g = prob.g_nodal()
    hier = O.build_hierarchy(2, prob.coarse_cells, refinements)
    ctx = threadpool_limits(1) if threadpool_limits else None
    times = []
    try:
        if ctx is not None:
            ctx.__enter__()
        for _ in range(repeats):
            t0 = time.perf_counter()
            O.fmg(hier, g, prob.f, prob.a, keep_levels=False)
            times.append(time.perf_counter() - t0)
    finally:
        if ctx is not None:
            ctx.__exit__(None, None, None)
    return prob.fine_dofs, times


def cpu_baseline(refinements: int = 7, repeats: int = 5):
    dofs, times = oracle_sample(refinements, repeats)
    t = statistics.median(times)
    return {"value": dofs / t, "unit": "DOF/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 numpy/scipy oracle FMG of the same problem family at 7 refinements "
                      f"({dofs} fine DOFs, 1/4 of the workload), median of {repeats} solves, hierarchy "
                      f"assembly excluded, BLAS limited to 1 thread"}


def run_reference(args):
    import torch

    dist, world, rank, _ = dist_setup(torch)
    if rank != 0:
        return
    dofs, times = oracle_sample(7, args.warmup + args.steps)
    t = statistics.mean(times[args.warmup:]) if args.steps > 0 else statistics.mean(times)
    v = dofs / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "7 refinements (1,046,529 fine DOFs) per step"},
            "cpu_baseline": {"value": v, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                             "sample": "FP64 oracle FMG at 7 refinements of the workload's problem family"},
            "e2e": {"value": v, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- GPU arm

def time_solver(torch, fmg, solver, flush, steps, warmup):
    for _ in range(warmup):
        fmg.fmg_solve(solver.ctx, None, None)
    fmg.fmg_sync(solver.ctx, fmg.fmg_stats())
    ms = []
    for _ in range(steps):
        with torch.cuda.stream(solver.stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(solver.stream)
        fmg.fmg_solve(solver.ctx, None, None)
        e1.record(solver.stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    fmg.fmg_sync(solver.ctx, fmg.fmg_stats())
    return ms


def kernel_times(torch, fmg, solver, flush, steps, level):
    """Instrumented solves: per-kind durations on the finest level (CUDA events in the graph)."""
    fmg.fmg_set_kernel_timing(solver.ctx, True)
    fmg.fmg_solve(solver.ctx, None, fmg.fmg_stats())
    acc = {fmg.KT_AUGMENTED: [0.0, 0], fmg.KT_SMOOTH_TOP: [0.0, 0], fmg.KT_CORRECTION: [0.0, 0]}
    for _ in range(steps):
        with torch.cuda.stream(solver.stream):
            flush.zero_()
        fmg.fmg_solve(solver.ctx, None, None)
        for kind in acc:
            t, n = fmg.fmg_kernel_time(solver.ctx, kind, level)
            acc[kind][0] += t
            acc[kind][1] += n
    fmg.fmg_set_kernel_timing(solver.ctx, False)
    return {k: (v[0] / max(v[1], 1), v[1]) for k, v in acc.items()}


def log(msg):
    if os.environ.get("FMG_BENCH_VERBOSE"):
        print(f"[bench] {msg}", file=sys.stderr, flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__

    dist, world, rank, local = dist_setup(torch)
    assert torch.cuda.is_available(), "the GPU arm needs a CUDA device"
    torch.cuda.set_device(local)
    __graft_entry__.build()
    from paper_1611_05677_gb300 import fmg, workloads as W

    prob = W.config_large_2d(seed=rank, refinements=args.refinements)
    g = prob.g_nodal()
    dofs = prob.fine_dofs
    n = prob.n_fine
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    hbm_peak, peak_kind = peaks()

    results = {}
    solvers = {}
    log("creating solvers")
    for prec in ("mixed", "fp64"):
        s = fmg.Solver(fmg.make_params(prob, precision=prec), g)
        st = fmg.fmg_stats()
        s.solve(stats=st)
        solvers[prec] = s
        results[prec] = {"stats": st}

    # ---- timed region (both precisions; clocks sampled throughout)
    log("timed region")
    barrier(dist, torch)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for prec in ("mixed", "fp64"):
            ms = time_solver(torch, fmg, solvers[prec], flush, args.steps, args.warmup)
            results[prec]["ms"] = ms
    torch.cuda.synchronize()
    barrier(dist, torch)
    launches_per_solve = fmg.fmg_graph_kernels(solvers["mixed"].ctx)
    for prec in ("mixed", "fp64"):
        mean_ms = statistics.mean(results[prec]["ms"])
        results[prec]["mean_ms"] = max_over_ranks(dist, torch, mean_ms)

    # ---- accuracy of both results against the exact solution and each other
    log("accuracy")
    us = prob.u_star()
    acc = {}
    outs = {}
    for prec in ("mixed", "fp64"):
        u = solvers[prec].solve().cpu().numpy()
        outs[prec] = u
        acc[prec] = float(math.sqrt(np.sum((u - us) ** 2) / n ** 2))
    diff = float(math.sqrt(np.sum((outs["mixed"] - outs["fp64"]) ** 2) / n ** 2))

    # ---- per-kernel durations (instrumented graph), finest level
    log("kernel timing")
    top = prob.levels
    kt = kernel_times(torch, fmg, solvers["mixed"], flush, max(3, args.steps // 2), top)
    smooth_ms, smooth_n = kt[fmg.KT_SMOOTH_TOP]
    aug_ms, aug_n = kt[fmg.KT_AUGMENTED]
    # algorithmic bytes of one FP32 red-black sweep: read b, read u, write u (4 B each) per node
    nodes = (n + 1) ** 2
    sweep_bytes = 12.0 * nodes
    smooth_gbs = sweep_bytes / (smooth_ms * 1e-3) / 1e9 if smooth_ms > 0 else None
    # augmented kernel at the top level: FP64 flops per launch (counted per fine node and pass)
    iters = int(results["mixed"]["stats"].newton_iters[top - 1])
    aug_flops = (40.0 * iters + 24.0) * dofs
    aug_tflops = aug_flops / (aug_ms * 1e-3) / 1e12 if aug_ms > 0 else None
    shares = {"augmented": aug_ms * aug_n, "smooth_top": smooth_ms * smooth_n}
    roof_smooth = {"kernel": "rbgs sweep (FP32, both colours) on the finest level", "bound": "hbm",
                   "achieved": smooth_gbs, "peak": hbm_peak, "unit": "GB/s",
                   "frac": (smooth_gbs / hbm_peak) if smooth_gbs else None, "traffic": None,
                   "peak_source": peak_kind, "avg_launch_ms": smooth_ms, "launches": smooth_n,
                   "algorithmic_bytes_per_launch": sweep_bytes}
    roof_aug = {"kernel": "augmented Newton (FP64) on the finest level", "bound": "alu",
                "achieved": aug_tflops, "peak": FP64_FLOPS_PEAK_DERIVED / 1e12, "unit": "TFLOP/s",
                "frac": (aug_tflops * 1e12 / FP64_FLOPS_PEAK_DERIVED) if aug_tflops else None,
                "traffic": None, "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz",
                "avg_launch_ms": aug_ms, "launches": aug_n, "algorithmic_flops_per_launch": aug_flops}
    dominant = max(shares, key=shares.get)
    roofline = roof_aug if dominant == "augmented" else roof_smooth
    other = roof_smooth if dominant == "augmented" else roof_aug

    # ---- end to end through the public API with host buffers (pinned)
    log("e2e")
    g_host = torch.from_numpy(np.ascontiguousarray(g)).pin_memory()
    out_host = torch.empty(g.shape, dtype=torch.float64).pin_memory()
    s = solvers["mixed"]
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fmg.fmg_set_rhs(s.ctx, g_host)
        fmg.fmg_solve(s.ctx, out_host, None)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_mean = max_over_ranks(dist, torch, statistics.mean(e2e_ms))

    cpu = None
    log("cpu baseline")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        mix = results["mixed"]["mean_ms"]
        f64 = results["fp64"]["mean_ms"]
        line = {
            "metric": METRIC,
            "value": world * dofs / (mix * 1e-3),
            "unit": "DOF/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": mix,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 cycles + f64 residual/Newton",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "mixed", "instances": world,
                       "global_batch": world, "seq_len": None, "parallelism": f"independent instances x{world}",
                       "l2": "flushed between steps (512 MB write outside the timed events)",
                       "m": 2, "nu": [2, 2], "p": 1},
            "fp64": {"value": world * dofs / (f64 * 1e-3), "unit": "DOF/s", "ms_per_step": f64,
                     "speedup_mixed_over_fp64": f64 / mix},
            "accuracy": {"l2_err_vs_exact_mixed": acc["mixed"], "l2_err_vs_exact_fp64": acc["fp64"],
                         "l2_diff_mixed_fp64": diff,
                         "newton_iters": list(results["mixed"]["stats"].newton_iters[:top]),
                         "flags": int(results["mixed"]["stats"].flags)},
            "roofline": roofline,
            "roofline_other": other,
            "cpu_baseline": cpu,
            "e2e": {"value": world * dofs / (e2e_mean * 1e-3), "unit": "DOF/s", "ms_per_step": e2e_mean,
                    "h2d_bytes_per_step": int(g.nbytes), "d2h_bytes_per_step": int(g.nbytes),
                    "path": "fmg_set_rhs(pinned host g) + fmg_solve(pinned host u_out)"},
            "gpu_launches": launches_per_solve * args.steps * 2,
            "gpu_launches_per_solve": launches_per_solve,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    for s in solvers.values():
        s.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the full multigrid solve for -Laplace(u) + u^3 = g (Algorithm 3.2).

Workload: 2D unit square, P1 on the right-triangle mesh, coarse H = 1/8, 8 uniform
refinements (2049 x 2049 nodes, 4,190,209 fine DOFs), u* = 8 seeded sin modes
(k, l in 1..6, N(0,1) amplitudes; seed = rank), m = 2 V(2,2) cycles, p = 1.

One step = one fmg_solve of that problem (level-1 Newton, every level's prolongation,
linearized right-hand side, V-cycles, augmented-space Newton and update) with the inputs
resident in HBM.  `value` is fine DOFs/s of the mixed-precision path (FP32 cycles inside a
float-float defect correction); the FP64 path is timed beside it ("fp64").  By default each path
uses its faster smoother at equal accuracy (mixed: Chebyshev-Jacobi with autotuned launch
shapes; FP64: red-black Gauss-Seidel).  L2 is flushed between steps (a 512 MB write outside
the timed events).

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
Under torchrun each rank solves its own instance (independent problems, weak scaling);
the reported time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
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
# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it stands, keyed by
# (kind, dim); a kernel changed since its capture has no entry (traffic null)
TRAFFIC = {("smooth_top", 2): 50_357_504 + 8_448,
           # the finest level's augmented Newton launch with its update kernel (2D), the Newton
           # launch alone (3D): dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture each
           ("augmented", 2): 68_331_008 + 1_463_040 + 33_567_488,
           ("augmented", 3): 579_506_944 + 128_349_184}
WORKLOAD = "2D unit square P1, H=1/8, 8 refinements (2049x2049 nodes, 4,190,209 fine DOFs), u^3, 8 sin modes"
WORKLOAD_3D = ("3D unit cube P1 on Kuhn tetrahedra, H=1/4, 6 refinements (257^3 nodes, 16,581,375 fine DOFs), "
               "exp(u)-1, 8 sin modes with U[0,1] amplitudes")


def solve_bytes_per_dof(dim: int, mixed: bool, m: int, smoother: str, nu=(2, 2), newton_passes: int = 3) -> float:
    """Compulsory HBM bytes per fine DOF of one FMG solve (Algorithm 3.2, p = 1), every pass
    streaming its arrays once.  A correction step on a level costs, per node: the right-hand
    side w (g - f(u)) of eq. (3.4) (24 B), m V-cycles, the augmented precompute (16 B),
    `newton_passes` Newton passes (8 B each) and the update (16 B).  A V-cycle costs, per node of
    its top level, its smoothing steps (red-black sweep 24 B in FP64 / 12 B in FP32; Chebyshev
    step 40 / 20 B), a residual + restriction and a prolongation + correction (16 + 8/2^d B each
    in FP64, half that in FP32), times the level sum 2^d / (2^d - 1); the mixed path adds its
    defect correction around each cycle (residual 20 B, update 20 B).  The FMG schedule
    multiplies a step by the same level sum."""
    ratio = 2 ** dim / (2 ** dim - 1)
    if mixed:
        sweep = 20.0 if smoother == "chebyshev" else 12.0
        transfer = 8 + 4 / 2 ** dim
        outer = 40.0
    else:
        sweep = 40.0 if smoother == "chebyshev" else 24.0
        transfer = 16 + 8 / 2 ** dim
        outer = 0.0
    cycle = outer + ((nu[0] + nu[1]) * sweep + 2 * transfer) * ratio
    step = 24 + m * cycle + 16 + newton_passes * 8 + 16
    return step * ratio


# FP64 operations (an FMA counts as two) per fine node of the FP64 path's augmented-space kernel
# for a u^3 (cubic) nonlinearity, counted from its per-node code: the first pass (f and f' at
# u~: 4; f - g: 1; the residual moments: 5; the Jacobian moments: 11; A u~ and the t, s moments:
# 11; the z counter: 1), each later Newton pass (U = alpha u~ + P c: 4; then 4 + 1 + 5 + 11 + 1)
# and the update (U: 4, z: 1).
AUG64_FLOPS_FIRST = 33
AUG64_FLOPS_NEWTON = 26
AUG64_FLOPS_UPDATE = 5
# FP64 operations per node of one red-black sweep (both colours): 2D (4 neighbours summed: 3,
# + b: 1, * 1/4: 1), 3D (6 neighbours: 5, b * h + s: 2, * 1/6: 1)
RBGS64_FLOPS = {2: 5, 3: 8}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--refinements", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--single-solve", action="store_true",
                    help="build, create one solver and run one solve, then exit (for ncu captures)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="large2d", choices=["large2d", "3d", "batch", "serve"],
                    help="large2d: the headline single-instance solve; 3d: the 3D Kuhn-mesh solve (257^3); "
                         "batch: 256 independent instances; serve: a Poisson request stream through the server")
    ap.add_argument("--serve-count", type=int, default=2200)
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--max-inflight", type=int, default=8)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip tuning the launch shapes of the Chebyshev step kernel before timing")
    ap.add_argument("--smoother", default="auto", choices=["auto", "rbgs", "chebyshev"],
                    help="smoother of the multigrid cycles (large2d / 3d / batch); auto: each arm's faster one "
                         "at equal accuracy (Chebyshev for the mixed path, red-black for FP64)")
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

def oracle_sample(refinements: int, repeats: int, seed: int = 0, dim: int = 2, threads: int | None = 1,
                  prob=None):
    """FP64 oracle FMG on a bounded sample of the workload: same H, fewer refinements (or the
    given problem), BLAS limited to `threads` (None: every core)."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:  # pragma: no cover
        threadpool_limits = None
    from oracle import fmg_oracle as O
    from paper_1611_05677_gb300 import workloads as W

    if prob is None:
        prob = (W.config_large_2d(seed=seed, refinements=refinements) if dim == 2
                else W.config_3d(seed=seed, refinements=refinements))
    g = prob.g_nodal()
    hier = O.build_hierarchy(prob.dim, prob.coarse_cells, prob.refinements)
    ctx = threadpool_limits(threads) if threadpool_limits else None
    times = []
    try:
        if ctx is not None:
            ctx.__enter__()
        for _ in range(repeats):
            t0 = time.perf_counter()
            O.fmg(hier, g, prob.f, prob.a, m=prob.m_vcycles, keep_levels=False)
            times.append(time.perf_counter() - t0)
    finally:
        if ctx is not None:
            ctx.__exit__(None, None, None)
    return prob.fine_dofs, times


def host_cpu():
    """The host's core count and CPU model (from /proc/cpuinfo where it exists)."""
    import platform

    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in ln:
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model in ("", platform.machine()):
        try:   # Arm hosts: /proc/cpuinfo has no model name; lscpu decodes the part number
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name:"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def cpu_baseline(refinements: int = 7, repeats: int = 5, dim: int = 2):
    """The FP64 oracle on the host: one thread (the reported value), all cores (the oracle is
    sparse and mostly single-threaded, so this is close), and the small configuration."""
    from paper_1611_05677_gb300 import workloads as W

    dofs, times = oracle_sample(refinements, repeats, dim=dim)
    t = statistics.median(times)
    dofs_all, times_all = oracle_sample(refinements, repeats, dim=dim, threads=None)
    small = W.config_small_2d() if dim == 2 else W.config_3d(seed=0, refinements=2)
    dofs_s, times_s = oracle_sample(0, 20, prob=small)
    host = host_cpu()
    return {"value": dofs / t, "unit": "DOF/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 numpy/scipy oracle FMG of the same problem family at {refinements} refinements "
                      f"({dofs} fine DOFs), median of {repeats} solves, hierarchy assembly excluded, BLAS "
                      f"limited to 1 thread",
            "host": host,
            "all_cores": {"value": dofs_all / statistics.median(times_all), "unit": "DOF/s",
                          "threads": host["nproc"],
                          "note": "same solves with BLAS on every core; the sparse steps stay single-threaded"},
            "small_config": {"value": dofs_s / statistics.median(times_s), "unit": "DOF/s", "cores": 1,
                             "workload": small.name, "fine_dofs": dofs_s, "median_of": 20}}


def run_reference(args):
    import torch

    dist, world, rank, _ = dist_setup(torch)
    if rank != 0:
        return
    dofs, times = oracle_sample(7, args.warmup + args.steps)
    t = statistics.mean(times[args.warmup:]) if args.steps > 0 else statistics.mean(times)
    v = dofs / t
    host = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "7 refinements (1,046,529 fine DOFs) per step"},
            "cpu_baseline": {"value": v, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                             "sample": "FP64 oracle FMG at 7 refinements of the workload's problem family",
                             "host": host},
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
    acc = {fmg.KT_AUGMENTED: [0.0, 0], fmg.KT_PRE_TOP: [0.0, 0], fmg.KT_POST_TOP: [0.0, 0],
           fmg.KT_CORRECTION: [0.0, 0], fmg.KT_SMOOTH_TOP: [0.0, 0]}
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

    if args.workload == "3d":
        prob = W.config_3d(seed=rank, refinements=6 if args.refinements == 8 else args.refinements)
    else:
        prob = W.config_large_2d(seed=rank, refinements=args.refinements)
    dim = prob.dim
    # cycles per correction step: the workload's m (2 in 2D as in the paper's examples; 3 on the
    # cube, where m = 2 leaves an algebraic error above a tenth of the discretization error)
    if args.smoother == "auto":
        smoother = {"mixed": "chebyshev", "fp64": "rbgs"}
    else:
        smoother = {"mixed": args.smoother, "fp64": args.smoother}
    m_cycles = {p: prob.m_vcycles for p in smoother}
    g = prob.g_nodal()
    dofs = prob.fine_dofs
    n = prob.n_fine
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    hbm_peak, peak_kind = peaks()

    results = {}
    solvers = {}
    log("creating solvers")
    for prec in ("mixed", "fp64"):
        s = fmg.Solver(fmg.make_params(prob, precision=prec, smoother=smoother[prec], m_vcycles=m_cycles[prec]), g)
        if not args.no_autotune:
            fmg.fmg_autotune(s.ctx)
            fmg.fmg_autotune_augmented(s.ctx)
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

    def l2(e):
        return float(math.sqrt(np.sum(e * e) / n ** dim))

    acc = {}
    outs = {}
    for prec in ("mixed", "fp64"):
        u = solvers[prec].solve().cpu().numpy()
        outs[prec] = u
        acc[prec] = l2(u - us)
    diff = l2(outs["mixed"] - outs["fp64"])
    # "solved to discretization accuracy" (Theorem 3.2 read as e_alg <= 0.1 e_disc): the exact
    # discrete solution u_bar is the fixed point of the correction step, reached by the FP64
    # solve with 8 correction steps per level (checked against 12)
    ubar = {}
    for p_steps in (8, 12):
        sb = fmg.Solver(fmg.make_params(prob, precision="fp64", smoother="rbgs", m_vcycles=m_cycles["fp64"],
                                        p_corrections=p_steps), g)
        ubar[p_steps] = sb.solve().cpu().numpy()
        sb.close()
    e_disc = l2(ubar[8] - us)
    alg = {"e_disc": e_disc, "ubar_settled": l2(ubar[12] - ubar[8]) / e_disc,
           "ubar": "FP64 GPU solve, 8 correction steps per level (difference to 12 steps in ubar_settled, "
                   "relative to e_disc)"}
    for prec in ("mixed", "fp64"):
        alg[f"e_alg_{prec}"] = l2(outs[prec] - ubar[8])
        alg[f"e_alg_over_e_disc_{prec}"] = alg[f"e_alg_{prec}"] / e_disc

    # ---- per-kernel durations (instrumented graph), finest level
    log("kernel timing")
    top = prob.levels
    kt = kernel_times(torch, fmg, solvers["mixed"], flush, max(3, args.steps // 2), top)
    aug_ms, aug_n = kt[fmg.KT_AUGMENTED]
    nodes = (n + 1) ** dim
    # augmented Newton on the top level (mixed path, float-float level data): the first pass
    # reads u~ and g (16 B/node), each chord pass reads u~ (8 B/node), the update reads u~ and
    # writes u (16 B/node); the stencil neighbours of the first pass are cache hits
    newton_top = int(results["mixed"]["stats"].newton_iters[top - 1]) or 1
    aug_bytes = (32.0 + 8.0 * (newton_top - 1)) * nodes
    aug_gbs = aug_bytes / (aug_ms * 1e-3) / 1e9 if aug_ms > 0 else None
    shares = {"augmented": aug_ms * aug_n}
    roof = {
        "augmented": {"kernel": "k_augmented (mixed) on the finest level", "bound": "hbm",
                      "achieved": aug_gbs, "peak": hbm_peak, "unit": "GB/s",
                      "frac": (aug_gbs / hbm_peak) if aug_gbs else None,
                      "traffic": TRAFFIC.get(("augmented", dim)), "peak_source": peak_kind,
                      "avg_launch_ms": aug_ms, "launches": aug_n, "algorithmic_bytes_per_launch": aug_bytes,
                      "newton_iterations": newton_top},
    }
    if dim == 2 and smoother["mixed"] == "rbgs":
        pre_ms, pre_n = kt[fmg.KT_PRE_TOP]
        post_ms, post_n = kt[fmg.KT_POST_TOP]
        # fused pre-smoothing on the top level: reads b (4 B/node), writes the correction
        # (4 B/node) and the coarse b and u (8 B per coarse node = 2 B/node)
        pre_bytes = 10.0 * nodes
        # fused post-smoothing on the top level: reads the correction and b (8 B/node), the
        # coarse correction (1 B/node), read-modify-writes the iterate (8-byte slots: 16 B/node)
        post_bytes = 25.0 * nodes
        pre_gbs = pre_bytes / (pre_ms * 1e-3) / 1e9 if pre_ms > 0 else None
        post_gbs = post_bytes / (post_ms * 1e-3) / 1e9 if post_ms > 0 else None
        shares.update({"pre_top": pre_ms * pre_n, "post_top": post_ms * post_n})
        roof["pre_top"] = {"kernel": "k_pre2_fused on the finest level", "bound": "hbm", "achieved": pre_gbs,
                           "peak": hbm_peak, "unit": "GB/s", "frac": (pre_gbs / hbm_peak) if pre_gbs else None,
                           "traffic": TRAFFIC.get(("pre_top", dim)), "peak_source": peak_kind, "avg_launch_ms": pre_ms,
                           "launches": pre_n, "algorithmic_bytes_per_launch": pre_bytes}
        roof["post_top"] = {"kernel": "k_post2_fused (top) on the finest level", "bound": "hbm", "achieved": post_gbs,
                            "peak": hbm_peak, "unit": "GB/s", "frac": (post_gbs / hbm_peak) if post_gbs else None,
                            "traffic": TRAFFIC.get(("post_top", dim)), "peak_source": peak_kind,
                            "avg_launch_ms": post_ms, "launches": post_n, "algorithmic_bytes_per_launch": post_bytes}
    else:
        sm_ms, sm_n = kt[fmg.KT_SMOOTH_TOP]
        if smoother["mixed"] == "chebyshev":
            # one Chebyshev step in FP32: read u, b (and d after the first step), write the
            # new iterate and d = 16 / 20 B/node, 18 B/node on average over nu = 2 steps
            sm_bytes = 18.0 * nodes
            sm_kernel = f"k_cheb<float, {dim}> step on the finest level"
        else:
            # one red-black sweep (both colours) in FP32: read u and b, write u = 12 B/node
            sm_bytes = 12.0 * nodes
            sm_kernel = "k_rbgs3<float> sweep (both colours) on the finest level"
        sm_gbs = sm_bytes / (sm_ms * 1e-3) / 1e9 if sm_ms > 0 else None
        shares["smooth_top"] = sm_ms * sm_n
        roof["smooth_top"] = {"kernel": sm_kernel, "bound": "hbm",
                              "achieved": sm_gbs, "peak": hbm_peak, "unit": "GB/s",
                              "frac": (sm_gbs / hbm_peak) if sm_gbs else None,
                              "traffic": TRAFFIC.get(("smooth_top", dim)), "peak_source": peak_kind,
                              "avg_launch_ms": sm_ms, "launches": sm_n, "algorithmic_bytes_per_launch": sm_bytes}
    dominant = max(shares, key=shares.get)
    roofline = roof[dominant]
    other = {k: v for k, v in roof.items() if k != dominant}

    # ---- FP64 arm: its ALU-bound kernels against the measured FP64 FMA rate
    log("fp64 roofline")
    fp64_peak = fmg.fmg_fp64_fma_rate(10) / 1e12
    kt64 = kernel_times(torch, fmg, solvers["fp64"], flush, max(3, args.steps // 2), top)
    fp64_roof = {}
    interior = (n - 1) ** dim
    sw_ms, sw_n = kt64[fmg.KT_SMOOTH_TOP]
    if sw_ms > 0:
        tf = RBGS64_FLOPS[dim] * interior / (sw_ms * 1e-3) / 1e12
        fp64_roof["rbgs_sweep"] = {"kernel": f"k_rbgs{dim}<double> sweep (both colours) on the finest level",
                                   "bound": "fp64_alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s",
                                   "frac": tf / fp64_peak, "flops_per_node": RBGS64_FLOPS[dim],
                                   "avg_launch_ms": sw_ms, "launches": sw_n}
    a64_ms, a64_n = kt64[fmg.KT_AUGMENTED]
    its64 = int(results["fp64"]["stats"].newton_iters[top - 1]) or 1
    if a64_ms > 0 and prob.f == "cubic":
        fpn = AUG64_FLOPS_FIRST + AUG64_FLOPS_NEWTON * (its64 - 1) + AUG64_FLOPS_UPDATE
        tf = fpn * interior / (a64_ms * 1e-3) / 1e12
        fp64_roof["augmented"] = {"kernel": f"k_augmented<{dim}, 0> (FP64 path) on the finest level",
                                  "bound": "fp64_alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s",
                                  "frac": tf / fp64_peak, "flops_per_node": fpn, "newton_iterations": its64,
                                  "avg_launch_ms": a64_ms, "launches": a64_n}
    fp64_dom = max(fp64_roof, key=lambda k: fp64_roof[k]["avg_launch_ms"] * fp64_roof[k]["launches"]) \
        if fp64_roof else None
    fp64_roofline = dict(fp64_roof[fp64_dom]) if fp64_dom else None
    if fp64_roofline is not None:
        fp64_roofline["peak_source"] = ("measured: fmg_fp64_fma_rate, independent FP64 FMA chains on every SM "
                                        "(an FMA counts as two)")
        fp64_roofline["other"] = {k: v for k, v in fp64_roof.items() if k != fp64_dom}

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
        cpu = cpu_baseline() if dim == 2 else cpu_baseline(refinements=4, repeats=5, dim=3)

    if rank == 0:
        mix = results["mixed"]["mean_ms"]
        f64 = results["fp64"]["mean_ms"]
        # the whole solve against the HBM roofline: compulsory bytes of the method as run (its
        # smoother, m, nu = 2/2, three Newton passes per step) over the measured solve time
        solve_hbm = {"unit": "GB/s", "peak": hbm_peak, "peak_source": peak_kind,
                     "model": "compulsory bytes per fine DOF: per correction step 24 (rhs) + m V-cycles + 16 "
                              "(precompute) + 3 x 8 (Newton passes) + 16 (update), cycles and steps summed "
                              "over levels (x 2^d/(2^d-1)); each pass streams its arrays once"}
        for prec, ms in (("mixed", mix), ("fp64", f64)):
            bpd = solve_bytes_per_dof(dim, prec == "mixed", m_cycles[prec], smoother[prec])
            achieved = bpd * dofs / (ms * 1e-3) / 1e9
            solve_hbm[prec] = {"bytes_per_dof": bpd, "achieved": achieved, "frac": achieved / hbm_peak,
                               "ceiling_dofs_per_s": hbm_peak * 1e9 / bpd}
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
            "dtype": "f32 cycles + float-float (f32 pair) level data + f64 Newton",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if dim == 2 else WORKLOAD_3D, "precision": "mixed",
                       "smoother": smoother["mixed"], "fp64_smoother": smoother["fp64"], "instances": world,
                       "autotuned": not args.no_autotune,
                       "top_level_augmented_shape": {p: fmg.fmg_aug_shape(solvers[p].ctx, top) for p in solvers},
                       "top_level_cheb_shape": (fmg.fmg_tuned_shape(solvers["mixed"].ctx, top)
                                                if smoother["mixed"] == "chebyshev" else None),
                       "global_batch": world, "seq_len": None, "parallelism": f"independent instances x{world}",
                       "l2": "flushed between steps (512 MB write outside the timed events)",
                       "m": m_cycles["mixed"], "fp64_m": m_cycles["fp64"], "nu": [2, 2], "p": 1},
            "fp64": {"value": world * dofs / (f64 * 1e-3), "unit": "DOF/s", "ms_per_step": f64,
                     "speedup_mixed_over_fp64": f64 / mix, "roofline": fp64_roofline},
            "accuracy": {"l2_err_vs_exact_mixed": acc["mixed"], "l2_err_vs_exact_fp64": acc["fp64"],
                         "l2_diff_mixed_fp64": diff, "discretization": alg,
                         "newton_iters": list(results["mixed"]["stats"].newton_iters[:top]),
                         "flags": int(results["mixed"]["stats"].flags)},
            "roofline": roofline,
            "roofline_other": other,
            "solve_hbm": solve_hbm,
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


BATCH_WORKLOAD = ("batched: independent 2D P1 instances, H=1/4, refinements U{5..9}, a*u^3 with a~U[0.5,2], "
                  "seeded random-mode g; one CUDA graph, a branch per instance")


def prolong_2d(uc):
    """Nodal P1 interpolation onto the once-refined 2D mesh (right triangles split along the
    (0,0)-(1,1) diagonal; arrays x fastest): coincident nodes copy, edge midpoints average the
    edge's two ends."""
    import numpy as np

    nc = uc.shape[0] - 1
    uf = np.zeros((2 * nc + 1, 2 * nc + 1))
    uf[::2, ::2] = uc
    uf[::2, 1::2] = 0.5 * (uc[:, :-1] + uc[:, 1:])
    uf[1::2, ::2] = 0.5 * (uc[:-1, :] + uc[1:, :])
    uf[1::2, 1::2] = 0.5 * (uc[:-1, :-1] + uc[1:, 1:])
    return uf


def run_batch(args):
    """Batched solves: one step = one launch of the batch graph (every instance solved once)."""
    import numpy as np
    import torch

    import __graft_entry__

    dist, world, rank, local = dist_setup(torch)
    assert torch.cuda.is_available(), "the GPU arm needs a CUDA device"
    torch.cuda.set_device(local)
    __graft_entry__.build()
    from paper_1611_05677_gb300 import fmg, workloads as W

    probs = W.config_batch(seed=rank, count=args.batch_count)
    dofs = sum(p.fine_dofs for p in probs)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    # each precision on its faster smoother, as in the single-instance workloads
    if args.smoother == "auto":
        smoother = {"mixed": "chebyshev", "fp64": "rbgs"}
    else:
        smoother = {"mixed": args.smoother, "fp64": args.smoother}
    res = {}
    for prec in ("mixed", "fp64"):
        log(f"batch {prec}: creating {len(probs)} solvers")
        t0 = time.perf_counter()
        solvers = [fmg.Solver(fmg.make_params(p, precision=prec, smoother=smoother[prec]), p.g_nodal()) for p in probs]
        if not args.no_autotune and smoother[prec] == "chebyshev":
            # the launch-shape table is per level size: the deepest instance covers every level
            fmg.fmg_autotune(max(solvers, key=lambda s: s.params.refinements).ctx)
        batch = fmg.Batch(solvers, mode="phases")
        stats = batch.solve(wait=True)
        setup_s = time.perf_counter() - t0
        branches = fmg.Batch(solvers, mode="branches")
        branches.solve(wait=True)
        res[prec] = {"solvers": solvers, "batch": batch, "branches": branches, "setup_s": setup_s,
                     "flags": int(np.bitwise_or.reduce([st.flags for st in stats]))}

    def time_batch(b):
        for _ in range(args.warmup):
            b.solve()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            with torch.cuda.stream(b.stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            fmg.fmg_batch_solve(b.handle, None)
            e1.record(b.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return max_over_ranks(dist, torch, statistics.mean(ms))

    barrier(dist, torch)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for prec in ("mixed", "fp64"):
            res[prec]["ms"] = time_batch(res[prec]["batch"])
            res[prec]["branches_ms"] = time_batch(res[prec]["branches"])
    torch.cuda.synchronize()
    barrier(dist, torch)
    # one instance at a time (each instance's own graph), for comparison
    log("sequential")
    seq = {}
    for prec in ("mixed", "fp64"):
        solvers = res[prec]["solvers"]
        for s in solvers:
            fmg.fmg_solve(s.ctx, None, None)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        st = solvers[0].stream
        e0.record(st)
        for s in solvers:
            st.wait_stream(s.stream)
            s.stream.wait_stream(st)
            fmg.fmg_solve(s.ctx, None, None)
            st.wait_stream(s.stream)
        e1.record(st)
        e1.synchronize()
        seq[prec] = e0.elapsed_time(e1)
    # accuracy: the mixed results against the FP64 results, relative discrete L2 per instance
    # (the two arms' smoothers may differ, so this includes the algorithms' own difference)
    res["mixed"]["batch"].solve(wait=True)
    res["fp64"]["batch"].solve(wait=True)
    worst = 0.0
    for sm, sd in zip(res["mixed"]["solvers"], res["fp64"]["solvers"]):
        a = sm.solution().double()
        b = sd.solution().double()
        worst = max(worst, float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)))
    # "solved to discretization accuracy" on one instance per level count: e_alg = ||u - u_bar_h||
    # with u_bar_h the FP64 solve at 8 correction steps per level, against e_disc estimated by
    # Richardson as ||u_bar_h - P u_bar_2h|| / 3 (random-mode g has no exact solution)
    log("batch accuracy sample")
    alg = {}
    first = {}
    for i, p in enumerate(probs):
        first.setdefault(p.refinements, i)
    for r, i in sorted(first.items()):
        p = probs[i]
        ub = {}
        for rr in (r, r - 1):
            q = dataclasses.replace(p, refinements=rr)
            sb = fmg.Solver(fmg.make_params(q, precision="fp64", smoother="rbgs", p_corrections=8), q.g_nodal())
            ub[rr] = sb.solve().cpu().numpy()
            sb.close()
        n = p.n_fine
        l2 = lambda e: float(math.sqrt(np.sum(e * e) / n ** 2))
        e_disc = l2(ub[r] - prolong_2d(ub[r - 1])) / 3.0
        alg[f"r{r}"] = {prec: l2(res[prec]["solvers"][i].solution().cpu().numpy() - ub[r]) / e_disc
                        for prec in ("mixed", "fp64")}
    launches = res["mixed"]["batch"].kernel_nodes
    if rank == 0:
        mix, f64 = res["mixed"]["ms"], res["fp64"]["ms"]
        line = {
            "metric": METRIC, "value": world * dofs / (mix * 1e-3), "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mix, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 cycles + float-float (f32 pair) level data + f64 Newton",
            "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "instances": len(probs) * world, "fine_dofs_per_step": dofs,
                       "precision": "mixed", "l2": "flushed between steps (512 MB write outside the timed events)",
                       "parallelism": f"independent batches x{world}"},
            "fp64": {"value": world * dofs / (f64 * 1e-3), "unit": "DOF/s", "ms_per_step": f64,
                     "speedup_mixed_over_fp64": f64 / mix},
            "one_at_a_time": {"mixed_ms": seq["mixed"], "fp64_ms": seq["fp64"],
                              "batch_speedup_mixed": seq["mixed"] / mix},
            "layout": {"timed": "phases: one launch per phase over every instance that has the level",
                       "phase_launches_per_solve": {p: res[p]["batch"].kernel_nodes for p in ("mixed", "fp64")},
                       "phase_groups": {p: res[p]["batch"].groups for p in ("mixed", "fp64")},
                       "branches": {p: {"ms_per_step": res[p]["branches_ms"],
                                        "value": world * dofs / (res[p]["branches_ms"] * 1e-3),
                                        "launches_per_solve": res[p]["branches"].kernel_nodes}
                                    for p in ("mixed", "fp64")}},
            "smoother": smoother,
            "accuracy": {"max_rel_l2_diff_mixed_fp64": worst,
                         "e_alg_over_e_disc": alg,
                         "e_alg_over_e_disc_max": max(max(v.values()) for v in alg.values()),
                         "e_disc": "Richardson: ||u_bar_h - P u_bar_2h|| / 3, u_bar from FP64 solves with 8 "
                                   "correction steps per level; one instance per level count",
                         "flags": res["mixed"]["flags"] | res["fp64"]["flags"]},
            "setup_s": {p: res[p]["setup_s"] for p in ("mixed", "fp64")},
            "gpu_launches": launches * args.steps, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    for prec in ("mixed", "fp64"):
        res[prec]["batch"].close()
        res[prec]["branches"].close()
        for s in res[prec]["solvers"]:
            s.close()
    if dist is not None:
        dist.destroy_process_group()


SERVE_WORKLOAD = ("served: Poisson arrivals (mean 200 req/s), 70% 2D (refinements U{5..10} of H=1/4), 30% 3D "
                  "(U{3..6} of H=1/4), u^3 or exp(u)-1, random-mode g; mixed precision; request server with "
                  "continuous batching")


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def random_mode_g(p, out):
    """Writes the request's own random-mode g = sum_q c_q prod_ax sin(k_q,ax pi x_ax) on its nodal
    grid (x fastest) into the host tensor `out`, as one matrix product of the separable factors
    (the last axis' factors times the in-plane ones): milliseconds on the host cores even for a
    16.8M-node field."""
    import torch

    n = p.n_fine
    x = torch.arange(n + 1, dtype=torch.float64) / n
    outer, inner = [], []
    for kv, c in p.g_modes:
        sx = torch.sin(kv[0] * math.pi * x)
        if p.dim == 2:
            inner.append(sx)
            outer.append(float(c) * torch.sin(kv[1] * math.pi * x))
        else:
            inner.append(torch.outer(torch.sin(kv[1] * math.pi * x), sx).reshape(-1))
            outer.append(float(c) * torch.sin(kv[2] * math.pi * x))
    torch.mm(torch.stack(outer).T, torch.stack(inner), out=out.view(n + 1, -1))


def size_class(p):
    if p.dim == 2:
        return "2d_r5-7" if p.refinements <= 7 else "2d_r8-10"
    return "3d_r3-4" if p.refinements <= 4 else "3d_r5-6"


def run_serve(args):
    """Open-loop serving: requests submitted at their Poisson arrival times; then the same
    requests submitted at once (the server's capacity).  Every request carries its own seeded
    random-mode g, written into a pinned host buffer just before it is submitted (a ring of
    buffers per shape; a buffer is refilled only after the request that used it last has
    completed)."""
    import numpy as np
    import torch

    import __graft_entry__

    dist, world, rank, local = dist_setup(torch)
    assert torch.cuda.is_available(), "the GPU arm needs a CUDA device"
    torch.cuda.set_device(local)
    __graft_entry__.build()
    from paper_1611_05677_gb300 import fmg, workloads as W

    torch.set_num_threads(os.cpu_count() or 1)
    reqs = W.request_stream(seed=rank, count=args.serve_count, rate=args.serve_rate)
    ring = args.max_inflight + 4
    shapes = {}
    for _, p in reqs:
        shapes.setdefault((p.dim, p.refinements), (p.n_fine + 1,) * p.dim)
    log("allocating pinned rings")
    gbuf = {k: [torch.empty(v, dtype=torch.float64).pin_memory() for _ in range(ring)] for k, v in shapes.items()}
    ubuf = {k: [torch.empty(v, dtype=torch.float64).pin_memory() for _ in range(ring)] for k, v in shapes.items()}
    last = {k: [None] * ring for k in shapes}
    nxt = {k: 0 for k in shapes}
    params = [fmg.make_params(p, precision="mixed") for _, p in reqs]
    server = fmg.Server(max_inflight=args.max_inflight)
    gen_ms = []

    def collect(into):
        while True:
            rs = server.poll(256)
            if not rs:
                return
            for r in rs:
                into[r.ticket] = r

    def buffers(i, into):
        p = reqs[i][1]
        key = (p.dim, p.refinements)
        j = nxt[key]
        nxt[key] = (j + 1) % ring
        while last[key][j] is not None and last[key][j] not in into:
            collect(into)
            time.sleep(0.0002)
        t = time.perf_counter()
        random_mode_g(p, gbuf[key][j])
        gen_ms.append((time.perf_counter() - t) * 1e3)
        return key, j

    def submit(i, into, tickets):
        key, j = buffers(i, into)
        tk = server.submit(params[i], gbuf[key][j], ubuf[key][j])
        last[key][j] = tk
        tickets.append(tk)

    # ---- open loop at the arrival times
    log("open loop")
    done = {}
    tickets = []
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for i, (t_arr, p) in enumerate(reqs):
            while True:
                dt = t0 + t_arr - time.perf_counter()
                if dt <= 0:
                    break
                collect(done)
                time.sleep(min(dt, 0.0005))
            submit(i, done, tickets)
        server.drain(600.0)
        t_end = time.perf_counter()
        collect(done)
        # ---- closed loop: everything at once (capacity)
        log("burst")
        burst = dict(done)
        tb0 = time.perf_counter()
        btickets = []
        for i in range(args.serve_warmup, len(reqs)):
            submit(i, burst, btickets)
        server.drain(600.0)
        tb1 = time.perf_counter()
        collect(burst)
    info = server.info()
    measured = range(args.serve_warmup, len(reqs))
    lat = [done[tickets[i]].latency_ms for i in measured]
    que = [done[tickets[i]].queue_ms for i in measured]
    by_class = {}
    for i in measured:
        r = done[tickets[i]]
        c = by_class.setdefault(size_class(reqs[i][1]), {"lat": [], "queue": [], "service": []})
        c["lat"].append(r.latency_ms)
        c["queue"].append(r.queue_ms)
        c["service"].append(r.latency_ms - r.queue_ms)
    classes = {k: {"count": len(v["lat"]), "latency_p50": percentile(v["lat"], 0.5),
                   "latency_p99": percentile(v["lat"], 0.99), "queue_p50": percentile(v["queue"], 0.5),
                   "queue_p99": percentile(v["queue"], 0.99), "service_p50": percentile(v["service"], 0.5),
                   "service_p99": percentile(v["service"], 0.99)} for k, v in sorted(by_class.items())}
    bad = sum(1 for t in tickets if done[t].status != fmg.FMG_OK) + sum(
        1 for t in btickets if burst[t].status != fmg.FMG_OK)
    dofs = sum(reqs[i][1].fine_dofs for i in measured)
    span = t_end - (t0 + reqs[args.serve_warmup][0])
    server.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": world * dofs / span, "unit": "DOF/s", "n_gpus": world,
            "steps": len(measured), "warmup": args.serve_warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 cycles + float-float (f32 pair) level data + f64 Newton", "data": "synthetic",
            "config": {"workload": SERVE_WORKLOAD, "requests": len(reqs), "measured": len(measured),
                       "rate_per_s": args.serve_rate, "max_inflight": args.max_inflight,
                       "g": "each request's own seeded random-mode field, written on the host before its submit"},
            "latency_ms": {"p50": percentile(lat, 0.5), "p99": percentile(lat, 0.99), "max": max(lat),
                           "queue_p50": percentile(que, 0.5), "queue_p99": percentile(que, 0.99)},
            "latency_by_size": classes,
            "g_generation_ms": {"p50": percentile(gen_ms, 0.5), "p99": percentile(gen_ms, 0.99)},
            "served_dofs_per_s_open_loop": dofs / span,
            "offered_dofs_per_s": dofs / (reqs[-1][0] - reqs[args.serve_warmup][0]),
            "capacity_dofs_per_s_burst": dofs / (tb1 - tb0),
            "failed_requests": bad,
            "server": {"contexts_created": info.contexts_created, "contexts_evicted": info.contexts_evicted,
                       "bytes_held": info.bytes_held, "hbm_budget": info.hbm_budget},
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def single_solve(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_05677_gb300 import fmg, workloads as W

    if args.workload == "3d":
        prob = W.config_3d(refinements=6 if args.refinements == 8 else args.refinements)
    else:
        prob = W.config_large_2d(refinements=args.refinements)
    sm = "rbgs" if args.smoother == "auto" else args.smoother
    s = fmg.Solver(fmg.make_params(prob, precision=args.precision, smoother=sm, m_vcycles=prob.m_vcycles),
                   prob.g_nodal())
    st = fmg.fmg_stats()
    s.solve(stats=st)
    torch.cuda.synchronize()
    print(json.dumps({"single_solve": prob.name, "precision": args.precision, "smoother": sm,
                      "newton_iters": list(st.newton_iters[:prob.levels]), "flags": int(st.flags)}))
    s.close()


def main():
    args = parse()
    if args.single_solve:
        single_solve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

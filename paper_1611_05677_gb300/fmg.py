"""Python binding of the C ABI in include/fmg.h (argument marshalling only).

Every function named fmg_* here calls the C function of the same name in
libfmg_gb300.so; all arithmetic of the solver runs in the library's CUDA
kernels.  PyTorch is used only for device memory (the context workspace and
output tensors) and CUDA streams.  Importing the module does not need a GPU;
loading the library does, and fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_size_t, c_uint, c_void_p

import numpy as np

from . import build as _build

FMG_OK = 0
FMG_ERR_INVALID = 1
FMG_ERR_OOM = 2
FMG_ERR_NO_CONVERGENCE = 3
FMG_ERR_NONFINITE = 4
FMG_ERR_TIMEOUT = 5
FMG_ERR_CUDA = 6
STATUS_NAMES = {0: "FMG_OK", 1: "FMG_ERR_INVALID", 2: "FMG_ERR_OOM", 3: "FMG_ERR_NO_CONVERGENCE",
                4: "FMG_ERR_NONFINITE", 5: "FMG_ERR_TIMEOUT", 6: "FMG_ERR_CUDA"}

NONLIN = {"cubic": 0, "expm1": 1, "linear": 2, "signed_pow32": 3, "neg_exp_neg": 4}
PREC = {"fp64": 0, "mixed": 1}
SMOOTHER = {"rbgs": 0, "chebyshev": 1}
NONLINEAR = {"newton": 0, "fixed_point": 1}


class fmg_params(ctypes.Structure):
    _fields_ = [("dim", c_int), ("coarse_cells", c_int), ("refinements", c_int), ("f", c_int),
                ("f_scale", c_double), ("m_vcycles", c_int), ("nu_pre", c_int), ("nu_post", c_int),
                ("p_corrections", c_int), ("precision", c_int), ("newton_tol", c_double),
                ("newton_maxit", c_int), ("level1_tol", c_double), ("level1_maxit", c_int), ("smoother", c_int),
                ("nonlinear", c_int), ("coefficient", c_void_p)]


class fmg_stats(ctypes.Structure):
    _fields_ = [("levels", c_int), ("level1_iters", c_int), ("newton_iters", c_int * 32),
                ("alpha", c_double * 32), ("flags", c_uint)]


class fmg_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", c_size_t), ("max_inflight", c_int), ("poll_us", c_int)]


class fmg_server_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_ulonglong), ("status", c_int), ("stats", fmg_stats),
                ("queue_ms", c_double), ("latency_ms", c_double)]


class fmg_server_info(ctypes.Structure):
    _fields_ = [("hbm_budget", c_size_t), ("bytes_held", c_size_t), ("contexts_cached", c_int),
                ("in_flight", c_int), ("queued", c_int), ("submitted", c_size_t), ("completed", c_size_t),
                ("contexts_created", c_int), ("contexts_evicted", c_int)]


class FMGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
EXPORTS = ("fmg_default_params", "fmg_workspace_bytes", "fmg_create", "fmg_set_rhs", "fmg_solve", "fmg_sync",
           "fmg_solve_batch", "fmg_destroy", "fmg_last_error", "fmg_solution", "fmg_levels", "fmg_level_cells",
           "fmg_op_smooth", "fmg_op_smooth_f32", "fmg_op_residual", "fmg_op_vcycle", "fmg_op_correction_step",
           "fmg_op_level1_solve", "fmg_op_prolong", "fmg_set_kernel_timing", "fmg_kernel_time",
           "fmg_graph_kernels", "fmg_vcycle_noalloc", "fmg_debug_barrier_fault", "fmg_fp64_fma_rate",
           "fmg_batch_create", "fmg_batch_create_mode", "fmg_batch_info",
           "fmg_batch_solve", "fmg_batch_sync", "fmg_batch_destroy", "fmg_server_create", "fmg_server_submit", "fmg_server_poll", "fmg_server_drain",
           "fmg_server_get_info", "fmg_server_last_error", "fmg_server_destroy", "fmg_autotune", "fmg_tuned_shape",
           "fmg_autotune_augmented", "fmg_aug_shape")
KT_AUGMENTED = 0
KT_SMOOTH_TOP = 1
KT_CORRECTION = 2
KT_PRE_TOP = 3
KT_POST_TOP = 4


def library_path() -> str:
    return _build.LIB


def load():
    """Loads libfmg_gb300.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA solver library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = POINTER(fmg_params)
    S = POINTER(fmg_stats)
    sig = {
        "fmg_default_params": (None, [P]),
        "fmg_workspace_bytes": (c_int, [P, POINTER(c_size_t)]),
        "fmg_create": (c_int, [P, c_void_p, c_int, c_void_p, c_void_p, c_size_t, POINTER(c_void_p)]),
        "fmg_set_rhs": (c_int, [c_void_p, c_void_p, c_int]),
        "fmg_solve": (c_int, [c_void_p, c_void_p, c_int, S]),
        "fmg_sync": (c_int, [c_void_p, S]),
        "fmg_solve_batch": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p), S]),
        "fmg_destroy": (c_int, [c_void_p]),
        "fmg_last_error": (c_char_p, [c_void_p]),
        "fmg_solution": (c_void_p, [c_void_p]),
        "fmg_levels": (c_int, [c_void_p]),
        "fmg_level_cells": (c_int, [c_void_p, c_int]),
        "fmg_op_smooth": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int]),
        "fmg_op_smooth_f32": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int]),
        "fmg_op_residual": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
        "fmg_op_vcycle": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int]),
        "fmg_op_correction_step": (c_int, [c_void_p, c_int, c_void_p, S]),
        "fmg_op_level1_solve": (c_int, [c_void_p, c_void_p, S]),
        "fmg_op_prolong": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
        "fmg_set_kernel_timing": (c_int, [c_void_p, c_int]),
        "fmg_kernel_time": (c_int, [c_void_p, c_int, c_int, POINTER(c_double), POINTER(c_int)]),
        "fmg_graph_kernels": (c_int, [c_void_p]),
        "fmg_vcycle_noalloc": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
        "fmg_debug_barrier_fault": (c_int, [c_void_p, ctypes.c_longlong, c_int]),
        "fmg_fp64_fma_rate": (c_int, [c_int, POINTER(c_double)]),
        "fmg_batch_create": (c_int, [POINTER(c_void_p), c_int, c_void_p, POINTER(c_void_p)]),
        "fmg_batch_create_mode": (c_int, [POINTER(c_void_p), c_int, c_void_p, c_int, c_int, POINTER(c_void_p)]),
        "fmg_batch_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
        "fmg_batch_solve": (c_int, [c_void_p, S]),
        "fmg_batch_sync": (c_int, [c_void_p]),
        "fmg_batch_destroy": (c_int, [c_void_p]),
        "fmg_server_create": (c_int, [POINTER(fmg_server_config), POINTER(c_void_p)]),
        "fmg_server_submit": (c_int, [c_void_p, P, c_void_p, c_void_p, POINTER(ctypes.c_ulonglong)]),
        "fmg_server_poll": (c_int, [c_void_p, POINTER(fmg_server_result), c_int]),
        "fmg_server_drain": (c_int, [c_void_p, c_double]),
        "fmg_server_get_info": (c_int, [c_void_p, POINTER(fmg_server_info)]),
        "fmg_server_last_error": (c_char_p, []),
        "fmg_server_destroy": (c_int, [c_void_p]),
        "fmg_autotune": (c_int, [c_void_p, POINTER(c_int)]),
        "fmg_tuned_shape": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int)]),
        "fmg_autotune_augmented": (c_int, [c_void_p, POINTER(c_int)]),
        "fmg_aug_shape": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _device_sync():
    """Orders caller-side torch work before a synchronous component call."""
    import sys

    torch = sys.modules.get("torch")
    if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
        torch.cuda.synchronize()


def _check(status: int, ctx=None):
    if status != FMG_OK:
        msg = _lib.fmg_last_error(ctx)
        raise FMGError(status, msg.decode() if msg else "")


def _ptr(x):
    """(address, on_device) of a torch tensor, numpy array or raw int pointer (device)."""
    if x is None:
        return None, 1
    if isinstance(x, int):
        return x, 1
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data, 0
    # torch tensor
    assert x.is_contiguous()
    return x.data_ptr(), int(x.is_cuda)


# ---------------------------------------------------------------------------- C ABI, same names

def fmg_default_params() -> fmg_params:
    p = fmg_params()
    load().fmg_default_params(byref(p))
    return p


def fmg_workspace_bytes(p: fmg_params) -> int:
    n = c_size_t(0)
    _check(load().fmg_workspace_bytes(byref(p), byref(n)))
    return n.value


def fmg_create(p: fmg_params, g_fine, stream=None, workspace=None, workspace_bytes: int = 0):
    lib = load()
    gp, gdev = _ptr(g_fine)
    wp = None
    if workspace is not None:
        wp, _ = _ptr(workspace)
    ctx = c_void_p()
    _check(lib.fmg_create(byref(p), gp, gdev, stream, wp, workspace_bytes, byref(ctx)))
    return ctx


def fmg_set_rhs(ctx, g_fine):
    gp, gdev = _ptr(g_fine)
    _check(load().fmg_set_rhs(ctx, gp, gdev), ctx)


def fmg_solve(ctx, u_out=None, stats: fmg_stats | None = None):
    up, udev = _ptr(u_out)
    _check(load().fmg_solve(ctx, up, udev, byref(stats) if stats is not None else None), ctx)


def fmg_sync(ctx, stats: fmg_stats | None = None):
    _check(load().fmg_sync(ctx, byref(stats) if stats is not None else None), ctx)


def fmg_solve_batch(ctxs, u_outs=None, stats=None):
    arr = (c_void_p * len(ctxs))(*[c.value for c in ctxs])
    outs = None
    if u_outs is not None:
        outs = (c_void_p * len(ctxs))(*[_ptr(u)[0] for u in u_outs])
    st = (fmg_stats * len(ctxs))() if stats is None else stats
    _check(load().fmg_solve_batch(arr, len(ctxs), outs, st))
    return st


def fmg_destroy(ctx):
    if ctx is not None and ctx.value:
        load().fmg_destroy(ctx)


def fmg_last_error(ctx=None) -> str:
    r = load().fmg_last_error(ctx)
    return r.decode() if r else ""


def fmg_solution(ctx) -> int:
    return load().fmg_solution(ctx)


def fmg_levels(ctx) -> int:
    return load().fmg_levels(ctx)


def fmg_level_cells(ctx, level: int) -> int:
    return load().fmg_level_cells(ctx, level)


def fmg_op_smooth(ctx, level, b, u, sweeps, order=0):
    _device_sync()
    _check(load().fmg_op_smooth(ctx, level, _ptr(b)[0], _ptr(u)[0], sweeps, order), ctx)


def fmg_op_smooth_f32(ctx, level, b, u, sweeps, order=0):
    _device_sync()
    _check(load().fmg_op_smooth_f32(ctx, level, _ptr(b)[0], _ptr(u)[0], sweeps, order), ctx)


def fmg_op_residual(ctx, level, b, u, r):
    _device_sync()
    _check(load().fmg_op_residual(ctx, level, _ptr(b)[0], _ptr(u)[0], _ptr(r)[0]), ctx)


def fmg_op_vcycle(ctx, level, b, u, cycles=1):
    _device_sync()
    _check(load().fmg_op_vcycle(ctx, level, _ptr(b)[0], _ptr(u)[0], cycles), ctx)


def fmg_op_correction_step(ctx, level, u, stats: fmg_stats | None = None):
    _device_sync()
    _check(load().fmg_op_correction_step(ctx, level, _ptr(u)[0], byref(stats) if stats is not None else None), ctx)


def fmg_op_level1_solve(ctx, u, stats: fmg_stats | None = None):
    _device_sync()
    _check(load().fmg_op_level1_solve(ctx, _ptr(u)[0], byref(stats) if stats is not None else None), ctx)


def fmg_op_prolong(ctx, level, u_coarse, u_fine):
    _device_sync()
    _check(load().fmg_op_prolong(ctx, level, _ptr(u_coarse)[0], _ptr(u_fine)[0]), ctx)


def fmg_set_kernel_timing(ctx, on: bool):
    _check(load().fmg_set_kernel_timing(ctx, int(bool(on))), ctx)


def fmg_kernel_time(ctx, kind: int, level: int = 0):
    """(total milliseconds, launches) of one instrumented kernel kind in the last solve."""
    ms = c_double(0.0)
    n = c_int(0)
    _check(load().fmg_kernel_time(ctx, kind, level, byref(ms), byref(n)), ctx)
    return ms.value, n.value


def fmg_graph_kernels(ctx) -> int:
    return load().fmg_graph_kernels(ctx)


def fmg_debug_barrier_fault(ctx, spins: int = 0, skip_block: int = -1):
    """Failure-detection test hook: grid-barrier poll limit and a block that skips its first arrival."""
    _check(load().fmg_debug_barrier_fault(ctx, spins, skip_block), ctx)


def fmg_fp64_fma_rate(reps: int = 20) -> float:
    """The device's FP64 FMA rate in FLOP/s (an FMA counts as two), measured by the library."""
    r = c_double(0.0)
    _check(load().fmg_fp64_fma_rate(reps, byref(r)))
    return r.value


def fmg_vcycle_noalloc(dim, coarse_cells, level, b, u, cycles=1, nu_pre=2, nu_post=2, stream=None):
    """V-cycles with no device allocation (scratch in a fixed device array of the library).

    b and u must be contiguous float64 CUDA tensors of (coarse_cells 2^(level-1) + 1)^dim
    elements each (the level's nodal layout); anything else is rejected before the C call, so
    that no kernel ever sees a buffer of the wrong size, type or memory space.  The work is
    queued on `stream` (a torch.cuda.Stream, a raw cudaStream_t handle, or None for the legacy
    default stream) after the caller's current torch stream, and the call returns without
    waiting for the device."""
    import torch

    if dim not in (2, 3) or coarse_cells < 1 or not 1 <= level <= 23:
        raise FMGError(FMG_ERR_INVALID, "bad dim, coarse_cells or level")
    nodes = ((coarse_cells << (level - 1)) + 1) ** dim
    for name, x in (("b", b), ("u", u)):
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise FMGError(FMG_ERR_INVALID, f"{name} must be a contiguous float64 CUDA tensor")
        if x.numel() != nodes:
            raise FMGError(FMG_ERR_INVALID, f"{name} has {x.numel()} elements; level {level} needs {nodes}")
    if isinstance(stream, torch.cuda.Stream):
        run_on = stream
    elif stream is None:
        run_on = None
    else:
        run_on = torch.cuda.ExternalStream(int(stream))
    # order the caller's queued work (which produced b and u) before the cycles, by stream
    # order rather than a device-wide synchronization
    if run_on is not None:
        run_on.wait_stream(torch.cuda.current_stream())
    elif torch.cuda.current_stream().cuda_stream != 0:
        torch.cuda.current_stream().synchronize()
    sp = None if run_on is None else run_on.cuda_stream
    _check(load().fmg_vcycle_noalloc(dim, coarse_cells, level, b.data_ptr(), u.data_ptr(), cycles, nu_pre, nu_post,
                                     sp))


BATCH_AUTO, BATCH_PHASES, BATCH_BRANCHES = 0, 1, 2
_BATCH_MODES = {"auto": BATCH_AUTO, "phases": BATCH_PHASES, "branches": BATCH_BRANCHES}


def fmg_batch_create(ctxs, stream=None):
    arr = (c_void_p * len(ctxs))(*[c.value for c in ctxs])
    out = c_void_p()
    _check(load().fmg_batch_create(arr, len(ctxs), getattr(stream, "cuda_stream", stream), byref(out)))
    return out


def fmg_batch_create_mode(ctxs, stream=None, mode="auto", phase_split=0):
    """mode: "auto", "phases" or "branches" (or the FMG_BATCH_* value); phase_split: phase groups
    per set of agreeing schedules (0: the library's default)."""
    arr = (c_void_p * len(ctxs))(*[c.value for c in ctxs])
    out = c_void_p()
    m = _BATCH_MODES[mode] if isinstance(mode, str) else int(mode)
    _check(load().fmg_batch_create_mode(arr, len(ctxs), getattr(stream, "cuda_stream", stream), m, int(phase_split),
                                        byref(out)))
    return out


def fmg_batch_info(batch):
    """(mode, kernel nodes per solve, phase groups) of a batch; mode is "phases" or "branches"."""
    m, k, g = c_int(), c_int(), c_int()
    _check(load().fmg_batch_info(batch, byref(m), byref(k), byref(g)))
    return {BATCH_PHASES: "phases", BATCH_BRANCHES: "branches"}.get(m.value, "?"), k.value, g.value


def fmg_batch_solve(batch, stats=None):
    """Launches the batch; with stats (an array of fmg_stats, e.g. (fmg_stats * n)()) it waits."""
    _check(load().fmg_batch_solve(batch, stats))


def fmg_batch_sync(batch):
    _check(load().fmg_batch_sync(batch))


def fmg_batch_destroy(batch):
    if batch is not None and batch.value:
        load().fmg_batch_destroy(batch)


def _check_server(status: int):
    if status != FMG_OK:
        msg = _lib.fmg_server_last_error()
        raise FMGError(status, msg.decode() if msg else "")


def fmg_autotune(ctx) -> int:
    """Tunes the launch shapes of the context's stencil kernels; returns the levels tuned."""
    n = c_int(0)
    _check(load().fmg_autotune(ctx, byref(n)), ctx)
    return n.value


def fmg_tuned_shape(ctx, level: int):
    block, strip = c_int(0), c_int(0)
    _check(load().fmg_tuned_shape(ctx, level, byref(block), byref(strip)), ctx)
    return block.value, strip.value


def fmg_autotune_augmented(ctx) -> int:
    """Tunes the augmented Newton kernel's launch shape per level (changes rounding, see the
    header); returns the number of levels tuned."""
    n = c_int()
    _check(load().fmg_autotune_augmented(ctx, byref(n)), ctx)
    return n.value


def fmg_aug_shape(ctx, level: int):
    """(chunk length, blocks per coarse cell) of the augmented kernel on `level`."""
    a, b = c_int(), c_int()
    _check(load().fmg_aug_shape(ctx, level, byref(a), byref(b)), ctx)
    return a.value, b.value


def fmg_server_last_error() -> str:
    msg = load().fmg_server_last_error()
    return msg.decode() if msg else ""


def fmg_server_create(hbm_budget: int = 0, max_inflight: int = 0, poll_us: int = 0):
    cfg = fmg_server_config(hbm_budget, max_inflight, poll_us)
    out = c_void_p()
    _check_server(load().fmg_server_create(byref(cfg), byref(out)))
    return out


def fmg_server_submit(server, params: fmg_params, g_host, u_host) -> int:
    """Queues a solve; g_host and u_host are host arrays (numpy or CPU torch tensors)."""
    gp, gdev = _ptr(g_host)
    up, udev = _ptr(u_host)
    if gdev or udev:
        raise FMGError(FMG_ERR_INVALID, "the server takes host buffers")
    t = ctypes.c_ulonglong()
    _check_server(load().fmg_server_submit(server, byref(params), gp, up, byref(t)))
    return t.value


def fmg_server_poll(server, max_results: int = 64):
    buf = (fmg_server_result * max_results)()
    n = load().fmg_server_poll(server, buf, max_results)
    return [buf[i] for i in range(n)]


def fmg_server_drain(server, timeout_s: float = 600.0):
    _check_server(load().fmg_server_drain(server, timeout_s))


def fmg_server_get_info(server) -> fmg_server_info:
    info = fmg_server_info()
    _check_server(load().fmg_server_get_info(server, byref(info)))
    return info


def fmg_server_destroy(server):
    if server is not None and server.value:
        load().fmg_server_destroy(server)


# ---------------------------------------------------------------------------- convenience

def make_params(problem=None, **kw) -> fmg_params:
    """fmg_params from a workloads.Problem (and/or keyword overrides)."""
    p = fmg_default_params()
    if problem is not None:
        p.dim = problem.dim
        p.coarse_cells = problem.coarse_cells
        p.refinements = problem.refinements
        p.f = NONLIN[problem.f]
        p.f_scale = problem.a
        p.m_vcycles = problem.m_vcycles
        p.nu_pre = problem.nu_pre
        p.nu_post = problem.nu_post
        p.p_corrections = problem.p_corrections
        if getattr(problem, "coefficient", None) is not None:
            kw.setdefault("coefficient", problem.coefficient)
    # the coefficient last: its size check reads dim and coarse_cells
    for k, v in sorted(kw.items(), key=lambda kv: kv[0] == "coefficient"):
        if k == "coefficient":
            # the (coarse_cells^dim, dim) table of A's diagonal per cell of T_H; the array is
            # kept with the params (fmg_create copies it)
            if v is None:
                p.coefficient = None
                p._coefficient = None
                continue
            arr = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
            if arr.size != (p.coarse_cells ** p.dim) * p.dim:
                raise FMGError(FMG_ERR_INVALID, "coefficient must hold coarse_cells^dim rows of dim entries")
            p._coefficient = arr
            p.coefficient = arr.ctypes.data
            continue
        if k == "f" and isinstance(v, str):
            v = NONLIN[v]
        if k == "precision" and isinstance(v, str):
            v = PREC[v]
        if k == "smoother" and isinstance(v, str):
            v = SMOOTHER[v]
        if k == "nonlinear" and isinstance(v, str):
            v = NONLINEAR[v]
        setattr(p, k, v)
    return p


class Solver:
    """One problem instance on the current CUDA device.

    The context's workspace is a torch uint8 tensor (PyTorch's caching
    allocator owns the memory); the solver's work is ordered on `stream` (a
    torch.cuda.Stream; default: a new stream of its own), and solve() orders it
    after the caller's current stream and the caller's stream after it.
    """

    def __init__(self, params: fmg_params, g_fine, stream=None):
        import torch

        self.params = params
        self.dim = params.dim
        self.n_fine = params.coarse_cells << params.refinements
        self.stream = stream if stream is not None else torch.cuda.Stream()
        nbytes = fmg_workspace_bytes(params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        if isinstance(g_fine, np.ndarray):
            g_fine = np.ascontiguousarray(g_fine, dtype=np.float64)
        self.stream.wait_stream(torch.cuda.current_stream())
        self.ctx = fmg_create(params, g_fine, self.stream.cuda_stream, self.workspace, nbytes)

    @property
    def shape(self):
        return (self.n_fine + 1,) * self.dim

    def solve(self, out=None, stats: fmg_stats | None = None):
        import torch

        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        self.stream.wait_stream(torch.cuda.current_stream())
        fmg_solve(self.ctx, out, stats)
        torch.cuda.current_stream().wait_stream(self.stream)
        out.record_stream(self.stream)
        return out

    def set_rhs(self, g_fine):
        import torch

        self.stream.wait_stream(torch.cuda.current_stream())
        if isinstance(g_fine, np.ndarray):
            g_fine = np.ascontiguousarray(g_fine, dtype=np.float64)
        fmg_set_rhs(self.ctx, g_fine)

    def solution(self):
        """The context's fine-level result as a float64 view into its workspace (no copy)."""
        import torch

        off = fmg_solution(self.ctx) - self.workspace.data_ptr()
        nbytes = 8 * int(np.prod(self.shape))
        if off < 0 or off + nbytes > self.workspace.numel():
            raise FMGError(FMG_ERR_INVALID, "solution does not lie in the workspace")
        return self.workspace[off:off + nbytes].view(torch.float64).view(self.shape)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            fmg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several Solver instances solved together in one CUDA graph.

    mode: "phases" (one launch per phase over all instances, 2D), "branches" (a branch per
    instance) or "auto" (phases where the schedules allow it).  solve() launches it after the
    caller's current stream and orders the caller's stream after it; results are each
    solver's solution().
    """

    def __init__(self, solvers, stream=None, mode="auto", phase_split=0):
        import torch

        self.solvers = list(solvers)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.handle = fmg_batch_create_mode([s.ctx for s in self.solvers], self.stream.cuda_stream, mode, phase_split)
        self.mode, self.kernel_nodes, self.groups = fmg_batch_info(self.handle)

    def solve(self, wait: bool = False):
        import torch

        self.stream.wait_stream(torch.cuda.current_stream())
        st = (fmg_stats * len(self.solvers))() if wait else None
        fmg_batch_solve(self.handle, st)
        torch.cuda.current_stream().wait_stream(self.stream)
        return list(st) if wait else None

    def close(self):
        if getattr(self, "handle", None) is not None:
            fmg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request server over the C ABI: submit() queues a solve with host buffers, poll() returns
    finished requests.  The buffers of a request are kept referenced until it is polled."""

    def __init__(self, hbm_budget: int = 0, max_inflight: int = 0, poll_us: int = 0):
        self.handle = fmg_server_create(hbm_budget, max_inflight, poll_us)
        self._pending = {}

    def submit(self, params: fmg_params, g_host, u_host) -> int:
        if isinstance(g_host, np.ndarray):
            g_host = np.ascontiguousarray(g_host, dtype=np.float64)
        t = fmg_server_submit(self.handle, params, g_host, u_host)
        self._pending[t] = (g_host, u_host)
        return t

    def poll(self, max_results: int = 64):
        out = fmg_server_poll(self.handle, max_results)
        for r in out:
            self._pending.pop(r.ticket, None)
        return out

    def drain(self, timeout_s: float = 600.0):
        fmg_server_drain(self.handle, timeout_s)

    def info(self) -> fmg_server_info:
        return fmg_server_get_info(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            fmg_server_destroy(self.handle)
            self.handle = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

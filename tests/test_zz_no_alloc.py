"""The no-allocation V-cycle entry point (fmg_vcycle_noalloc) against the context-based one.

fmg_vcycle_noalloc serves callers that cannot call cudaMalloc (an application's own memory
pool owns the device memory, or an allocation's device synchronization is not acceptable):
it keeps every coarser level in a fixed device array of the library.  Through the C ABI it
must give what fmg_op_vcycle gives on an FP64 context, call after call: each call starts
from the previous call's result, so stale contents of the shared array would show up.
This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_05677_gb300 import fmg as F

    F.load()
    return F


@pytest.mark.parametrize("dim,H,level", [(2, 4, 6), (2, 8, 5), (3, 4, 4)])
def test_noalloc_vcycle_matches_context_vcycle(fmg, dim, H, level):
    from paper_1611_05677_gb300 import workloads as W

    prob = W.Problem(dim=dim, coarse_cells=H, refinements=level - 1, f="cubic", modes=[((1,) * dim, 1.0)])
    ctx_solver = fmg.Solver(fmg.make_params(prob, precision="fp64"), prob.g_nodal())
    n = H << (level - 1)
    shape = (n + 1,) * dim
    rng = np.random.default_rng(21)
    interior = tuple(slice(1, n) for _ in range(dim))
    b = np.zeros(shape)
    u0 = np.zeros(shape)
    b[interior] = rng.standard_normal((n - 1,) * dim) / n ** dim
    u0[interior] = 0.1 * rng.standard_normal((n - 1,) * dim)
    bd = torch.tensor(b, device="cuda")
    u_ref = torch.tensor(u0, device="cuda")
    u_na = torch.tensor(u0, device="cuda")
    stream = torch.cuda.Stream()
    for call in range(2):
        fmg.fmg_op_vcycle(ctx_solver.ctx, level, bd, u_ref, 2)
        fmg.fmg_vcycle_noalloc(dim, H, level, bd, u_na, cycles=2, nu_pre=2, nu_post=2, stream=stream)
        stream.synchronize()
        ref = u_ref.cpu().numpy()
        got = u_na.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), f"call {call}"
    ctx_solver.close()


def test_noalloc_rejects_sizes_beyond_its_array(fmg):
    # a 2D level with 2048 cells per side needs more than the fixed array holds; the buffers
    # have that level's full size, so even a check that let the call through would launch on
    # arrays of the right extent
    b = torch.zeros((2049, 2049), dtype=torch.float64, device="cuda")
    u = torch.zeros((2049, 2049), dtype=torch.float64, device="cuda")
    with pytest.raises(fmg.FMGError) as ei:
        fmg.fmg_vcycle_noalloc(2, 4, 10, b, u, cycles=1)
    assert ei.value.status == fmg.FMG_ERR_INVALID
    assert "at most" in fmg.fmg_last_error()
    assert float(u.abs().max()) == 0.0


def test_noalloc_wrapper_rejects_wrong_buffers(fmg):
    # wrong element count, FP32 and host arrays never reach the C entry point
    n = 4 << 4
    good = torch.zeros((n + 1, n + 1), dtype=torch.float64, device="cuda")
    for bad in (torch.zeros(16, dtype=torch.float64, device="cuda"),
                torch.zeros((n + 1, n + 1), dtype=torch.float32, device="cuda"),
                torch.zeros((n + 1, n + 1), dtype=torch.float64)):
        with pytest.raises(fmg.FMGError) as ei:
            fmg.fmg_vcycle_noalloc(2, 4, 5, good, bad, cycles=1)
        assert ei.value.status == fmg.FMG_ERR_INVALID

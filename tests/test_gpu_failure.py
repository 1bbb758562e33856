"""Failure detection on the device without a GPU fault.

The augmented-space Newton kernel (eq. 3.6 on V_H + span{u~}) is one cooperative launch whose
blocks meet at a grid barrier after every fine-grid pass.  Its waits are bounded: a block polls
a limited number of times, then sets the timeout flag and an abort word and leaves.  The test
hook fmg_debug_barrier_fault lowers the poll limit and makes one block skip its first arrival
(chosen on the host), so the other blocks' waits run out: the solve must report
FMG_ERR_TIMEOUT with flag bit 4, and the same context must solve correctly -- bitwise as
before -- once the hook is off.  Nothing traps, faults or waits without bound.
"""
import numpy as np
import pytest

from paper_1611_05677_gb300 import workloads as W

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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_barrier_wait_runs_out_and_the_context_recovers(fmg, precision):
    prob = W.Problem(dim=2, coarse_cells=8, refinements=3, f="cubic", modes=[((1, 1), 1.0), ((2, 3), 0.5)])
    s = fmg.Solver(fmg.make_params(prob, precision=precision), prob.g_nodal())
    ref = s.solve().cpu().numpy()
    fmg.fmg_debug_barrier_fault(s.ctx, 4096, 1)
    st = fmg.fmg_stats()
    with pytest.raises(fmg.FMGError) as ei:
        s.solve(stats=st)
    assert ei.value.status == fmg.FMG_ERR_TIMEOUT
    assert st.flags & 16
    assert "timed out" in fmg.fmg_last_error(s.ctx)
    fmg.fmg_debug_barrier_fault(s.ctx, 0, -1)
    st = fmg.fmg_stats()
    u = s.solve(stats=st).cpu().numpy()
    assert st.flags == 0
    assert np.array_equal(u, ref)
    s.close()


def test_barrier_hook_rejects_bad_arguments(fmg):
    prob = W.Problem(dim=2, coarse_cells=4, refinements=2, f="cubic", modes=[((1, 1), 1.0)])
    s = fmg.Solver(fmg.make_params(prob), prob.g_nodal())
    for spins, skip in ((-1, -1), (0, -2)):
        with pytest.raises(fmg.FMGError) as ei:
            fmg.fmg_debug_barrier_fault(s.ctx, spins, skip)
        assert ei.value.status == fmg.FMG_ERR_INVALID
    s.close()

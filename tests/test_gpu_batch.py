"""Batched solves (one graph, a branch per instance, cluster Newton kernels) against solo solves
and the FP64 oracle.

Each instance of a batch is an independent Algorithm 3.2 run; batching only changes where
and how concurrently its kernels run (and the augmented-space Newton kernel's reduction
order: one partial per coarse cell instead of one per block).  So every instance must give
its solo result: within the FP64 bar on the FP64 path, and within the mixed path's bar (a
tenth of the discretization error of the FP64 method) on the mixed path.
"""
import numpy as np
import pytest

from oracle import fmg_oracle as O
from paper_1611_05677_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def fmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_05677_gb300 import fmg as F

    F.load()
    return F


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def mixed_problems():
    out = []
    for i, (dim, H, r, f) in enumerate([(2, 4, 5, "cubic"), (2, 8, 3, "expm1"), (2, 4, 2, "cubic"),
                                        (3, 4, 2, "expm1"), (2, 4, 4, "neg_exp_neg")]):
        modes = [((1,) * dim, 1.0), ((2,) + (1,) * (dim - 1), 0.4 - 0.1 * i)]
        out.append(W.Problem(dim=dim, coarse_cells=H, refinements=r, f=f, a=1.0, modes=modes))
    return out


def test_batch_fp64_equals_solo_and_oracle(fmg):
    probs = W.config_batch(seed=5, count=6, rmin=1, rmax=5)
    probs.append(W.Problem(dim=3, coarse_cells=4, refinements=2, f="cubic", modes=[((1, 1, 1), 1.0)]))
    probs.append(W.Problem(dim=2, coarse_cells=8, refinements=3, f="signed_pow32", modes=[((1, 2), 1.0)]))
    solvers = [fmg.Solver(fmg.make_params(p, precision="fp64"), p.g_nodal()) for p in probs]
    solo, solo_stats = [], []
    for s in solvers:
        st = fmg.fmg_stats()
        solo.append(s.solve(stats=st).cpu().numpy())
        solo_stats.append(st)
    batch = fmg.Batch(solvers)
    stats = batch.solve(wait=True)
    got = [s.solution().cpu().numpy() for s in solvers]
    for i, p in enumerate(probs):
        assert stats[i].flags == 0, p.name
        assert rel(got[i], solo[i]) <= FP64_TOL, p.name
        for k in range(1, p.levels + 1):
            assert abs(stats[i].newton_iters[k - 1] - solo_stats[i].newton_iters[k - 1]) <= 1, (p.name, k)
        if p.refinements <= 3:
            hier = O.build_hierarchy(p.dim, p.coarse_cells, p.refinements)
            res = O.fmg(hier, p.g_nodal(), p.f, p.a)
            ref = O.to_nodal(hier.level(p.refinements + 1), res.u[-1])
            assert rel(got[i], ref) <= FP64_TOL, p.name
    # a second launch of the same graph gives the same bits
    batch.solve(wait=True)
    again = [s.solution().cpu().numpy() for s in solvers]
    for a, b in zip(got, again):
        assert np.array_equal(a, b)
    # and the instances still solve on their own afterwards
    after = solvers[0].solve().cpu().numpy()
    assert np.array_equal(after, solo[0])
    batch.close()
    for s in solvers:
        s.close()


def test_batch_mixed_keeps_the_mixed_bar(fmg):
    probs = mixed_problems()
    solvers = [fmg.Solver(fmg.make_params(p, precision="mixed"), p.g_nodal()) for p in probs]
    batch = fmg.Batch(solvers)
    stats = batch.solve(wait=True)
    for i, p in enumerate(probs):
        assert stats[i].flags == 0, p.name
        hier = O.build_hierarchy(p.dim, p.coarse_cells, p.refinements)
        g = p.g_nodal()
        res = O.fmg(hier, g, p.f, p.a)
        lev = hier.level(p.refinements + 1)
        ub, _ = O.newton_full(lev, O.load_vector(lev, g), p.f, p.a, U0=res.u[-1])
        e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, p.u_star()))
        u = O.from_nodal(lev, solvers[i].solution().cpu().numpy())
        assert O.discrete_l2(lev, u - res.u[-1]) <= 0.1 * e_disc, p.name
    batch.close()
    for s in solvers:
        s.close()


def test_one_shot_solve_batch_writes_outputs(fmg):
    probs = W.config_batch(seed=9, count=3, rmin=2, rmax=4)
    solvers = [fmg.Solver(fmg.make_params(p, precision="fp64"), p.g_nodal()) for p in probs]
    solo = [s.solve().cpu().numpy() for s in solvers]
    outs = [torch.empty(s.shape, dtype=torch.float64, device="cuda") for s in solvers]
    torch.cuda.synchronize()
    st = fmg.fmg_solve_batch([s.ctx for s in solvers], outs)
    for i in range(len(probs)):
        assert st[i].flags == 0
        assert rel(outs[i].cpu().numpy(), solo[i]) <= FP64_TOL
    for s in solvers:
        s.close()


def test_contexts_of_different_sizes_in_any_order(fmg):
    # shared kernels keep the largest shared-memory limit any context asked for
    big = W.Problem(dim=2, coarse_cells=8, refinements=3, f="cubic", modes=[((1, 1), 1.0)])
    small = W.Problem(dim=2, coarse_cells=4, refinements=3, f="cubic", modes=[((1, 1), 1.0)])
    for prec in ("fp64", "mixed"):
        sb = fmg.Solver(fmg.make_params(big, precision=prec), big.g_nodal())
        ss = fmg.Solver(fmg.make_params(small, precision=prec), small.g_nodal())
        st = fmg.fmg_stats()
        sb.solve(stats=st)
        assert st.flags == 0
        ss.solve(stats=st)
        assert st.flags == 0
        sb.close()
        ss.close()

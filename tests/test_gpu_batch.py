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


def phase_problems(H=4, rs=(1, 4, 2, 5, 3, 4), seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for i, r in enumerate(rs):
        k = 1 + i % 3
        modes = [((1, 1), 1.0), ((k, 2), float(rng.uniform(-0.5, 0.5)))]
        out.append(W.Problem(dim=2, coarse_cells=H, refinements=r, f="cubic", a=float(rng.uniform(0.5, 2.0)),
                             modes=modes))
    return out


@pytest.mark.parametrize("prec,smoother", [("mixed", "chebyshev"), ("mixed", "rbgs"), ("fp64", "rbgs"),
                                           ("fp64", "chebyshev")])
def test_phase_batch_gives_the_branch_batch_bits(fmg, prec, smoother):
    # uneven level counts (1..5 refinements), per-instance a and g: one phase group whose
    # stages run every instance that still has the level; same kernels, same arguments per
    # instance as the branch layout, so the same bits and the same Newton counts
    probs = phase_problems()
    res = {}
    for mode in ("branches", "phases"):
        solvers = [fmg.Solver(fmg.make_params(p, precision=prec, smoother=smoother), p.g_nodal()) for p in probs]
        b = fmg.Batch(solvers, mode=mode, phase_split=1)
        assert b.mode == mode
        stats = b.solve(wait=True)
        res[mode] = ([s.solution().cpu().numpy() for s in solvers], stats, b.kernel_nodes, b.groups)
        # a second launch gives the same bits
        b.solve(wait=True)
        for s, u in zip(solvers, res[mode][0]):
            assert np.array_equal(s.solution().cpu().numpy(), u)
        b.close()
        for s in solvers:
            s.close()
    ub, sb, kb, _ = res["branches"]
    up, sp, kp, gp = res["phases"]
    assert gp == 1
    assert kp < kb   # one launch per phase instead of one per instance
    for i, p in enumerate(probs):
        assert sp[i].flags == 0, p.name
        assert np.array_equal(up[i], ub[i]), p.name
        assert list(sp[i].newton_iters[:p.levels]) == list(sb[i].newton_iters[:p.levels]), p.name


def test_phase_batch_fp64_matches_the_oracle(fmg):
    probs = phase_problems(rs=(3, 1, 2))
    solvers = [fmg.Solver(fmg.make_params(p, precision="fp64"), p.g_nodal()) for p in probs]
    b = fmg.Batch(solvers, mode="phases")
    stats = b.solve(wait=True)
    for i, p in enumerate(probs):
        assert stats[i].flags == 0
        hier = O.build_hierarchy(p.dim, p.coarse_cells, p.refinements)
        res = O.fmg(hier, p.g_nodal(), p.f, p.a)
        ref = O.to_nodal(hier.level(p.refinements + 1), res.u[-1])
        assert rel(solvers[i].solution().cpu().numpy(), ref) <= FP64_TOL, p.name
    b.close()
    for s in solvers:
        s.close()


def test_phase_batch_groups_by_schedule(fmg):
    # two coarse meshes (1/H = 4 and 8) cannot share launches: two groups, each a branch of
    # phases, and the results are the branch layout's
    probs = phase_problems(H=4, rs=(2, 3)) + phase_problems(H=8, rs=(1, 2), seed=3)
    res = {}
    for mode in ("branches", "phases"):
        solvers = [fmg.Solver(fmg.make_params(p, precision="mixed", smoother="chebyshev"), p.g_nodal())
                   for p in probs]
        b = fmg.Batch(solvers, mode=mode, phase_split=1)
        b.solve(wait=True)
        res[mode] = ([s.solution().cpu().numpy() for s in solvers], b.groups)
        b.close()
        for s in solvers:
            s.close()
    assert res["phases"][1] == 2
    for a, c in zip(res["phases"][0], res["branches"][0]):
        assert np.array_equal(a, c)


def test_phase_layout_refuses_3d_and_auto_falls_back(fmg):
    probs = phase_problems(rs=(2,)) + [W.Problem(dim=3, coarse_cells=4, refinements=1, f="cubic",
                                                 modes=[((1, 1, 1), 1.0)])]
    solvers = [fmg.Solver(fmg.make_params(p, precision="fp64"), p.g_nodal()) for p in probs]
    with pytest.raises(fmg.FMGError) as ei:
        fmg.Batch(solvers, mode="phases")
    assert "phase" in str(ei.value)
    b = fmg.Batch(solvers)   # auto: branches
    assert b.mode == "branches"
    stats = b.solve(wait=True)
    assert all(st.flags == 0 for st in stats)
    b.close()
    for s in solvers:
        s.close()


def test_phase_groups_split_into_parallel_branches(fmg):
    # the default deals one set of agreeing schedules into several groups of similar level
    # counts; each still gives every instance the same bits
    probs = phase_problems(rs=(4, 1, 3, 2, 4, 1, 3, 2, 5))
    solvers = [fmg.Solver(fmg.make_params(p, precision="mixed", smoother="chebyshev"), p.g_nodal()) for p in probs]
    ref = fmg.Batch(solvers, mode="branches")
    ref.solve(wait=True)
    want = [s.solution().cpu().numpy() for s in solvers]
    ref.close()
    for split, groups in ((3, 3), (0, 8), (64, 9)):
        b = fmg.Batch(solvers, mode="phases", phase_split=split)
        assert b.groups == groups
        stats = b.solve(wait=True)
        assert all(st.flags == 0 for st in stats)
        for s, u in zip(solvers, want):
            assert np.array_equal(s.solution().cpu().numpy(), u)
        b.close()
    for s in solvers:
        s.close()

"""The mixed path's float-float level data (through the C ABI) against the FP64 oracle.

During a mixed solve the level iterates, the right-hand sides of eq. (3.4) and g are
float-float pairs, and only the solve's last correction step writes the FP64 result.  These
tests cover the paths around that representation: the correction-step op on a mixed context
(FP64 in, float-float inside, FP64 out), p > 1 correction steps per level (only the first
starts from the coarser level's interpolation), and the level-1-only hierarchy (whose
level-1 solve is the result and must be written as FP64).  The bars are the mixed path's:
the FP32 cycles leave a relative difference of about 1e-7 to the FP64 method, far below the
discretization error.
"""
import numpy as np
import pytest

from oracle import fmg_oracle as O
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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def problem(dim, H, r, f):
    modes = [((1,) * dim, 1.0), ((2, 3, 1)[:dim], 0.5)]
    return W.Problem(dim=dim, coarse_cells=H, refinements=r, f=f, a=1.0, modes=modes)


@pytest.mark.parametrize("dim,H,r,kind", [(2, 4, 3, "cubic"), (2, 8, 2, "expm1"), (3, 4, 2, "cubic"),
                                          (2, 4, 3, "signed_pow32")])
def test_mixed_correction_step_op_matches_the_fp64_step(fmg, dim, H, r, kind):
    prob = problem(dim, H, r, kind)
    s = fmg.Solver(fmg.make_params(prob, precision="mixed"), prob.g_nodal())
    hier = O.build_hierarchy(dim, H, r)
    k = r + 1
    lev = hier.level(k)
    G = O.load_vector(lev, prob.g_nodal())
    ub, _ = O.newton_full(lev, G, kind, prob.a)
    u0 = ub + 0.05 * np.random.default_rng(11).standard_normal(ub.shape)
    ref, info = O.correction_step(hier, k, u0, G, kind, prob.a)
    ud = dev(O.to_nodal(lev, u0))
    st = fmg.fmg_stats()
    fmg.fmg_op_correction_step(s.ctx, k, ud, st)
    assert st.flags == 0
    out = ud.cpu().numpy()
    assert rel(O.from_nodal(lev, out), ref) <= 1e-5
    assert abs(st.alpha[k - 1] - info.alpha) <= 1e-5
    # the op returns FP64 values on the caller's layout: the boundary ring stays zero
    mask = np.ones(out.size, bool)
    mask[lev.interior] = False
    assert np.all(out.ravel()[mask] == 0.0)
    s.close()


@pytest.mark.parametrize("dim,H,r,kind,p", [(2, 4, 4, "cubic", 2), (3, 4, 2, "expm1", 3)])
def test_mixed_several_correction_steps_per_level(fmg, dim, H, r, kind, p):
    prob = problem(dim, H, r, kind)
    hier = O.build_hierarchy(dim, H, r)
    g = prob.g_nodal()
    res = O.fmg(hier, g, kind, prob.a, p=p)
    lev = hier.level(r + 1)
    ub, _ = O.newton_full(lev, O.load_vector(lev, g), kind, prob.a, U0=res.u[-1])
    e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star()))
    s = fmg.Solver(fmg.make_params(prob, precision="mixed", p_corrections=p), g)
    st = fmg.fmg_stats()
    u = O.from_nodal(lev, s.solve(stats=st).cpu().numpy())
    assert st.flags == 0
    assert O.discrete_l2(lev, u - res.u[-1]) <= 0.1 * e_disc
    s.close()


def test_mixed_level1_only_hierarchy_returns_fp64(fmg):
    prob = W.Problem(dim=2, coarse_cells=8, refinements=0, f="cubic", modes=[((1, 1), 1.0)])
    s = fmg.Solver(fmg.make_params(prob, precision="mixed"), prob.g_nodal())
    u = s.solve().cpu().numpy()
    lev = O.assemble_level(2, 8)
    ref, _ = O.newton_full(lev, O.load_vector(lev, prob.g_nodal()), "cubic", 1.0, tol=1e-6, direct="dense")
    assert rel(u, O.to_nodal(lev, ref)) <= 1e-9
    s.close()


def test_mixed_solves_repeat_bitwise_and_match_fp64(fmg):
    """Graph replays start every level from the coarser level's float-float data again: two
    solves give the same bits, and the result is the FP64 method's to the mixed bar."""
    prob = problem(2, 8, 4, "cubic")
    g = prob.g_nodal()
    sm = fmg.Solver(fmg.make_params(prob, precision="mixed"), g)
    s64 = fmg.Solver(fmg.make_params(prob, precision="fp64"), g)
    a = sm.solve().cpu().numpy()
    b = sm.solve().cpu().numpy()
    c = s64.solve().cpu().numpy()
    assert np.array_equal(a, b)
    assert rel(a, c) <= 1e-5
    sm.close()
    s64.close()

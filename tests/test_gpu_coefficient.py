"""Parity of the variable-coefficient path with the oracle.

The model problem of Sec. 2, eq. (2.1), with a diagonal SPD coefficient A(x) constant on each
cell of T_H (entries U[0.5, 2], contrast 4): every level's stiffness keeps the (2d+1)-point
pattern with a weight per mesh edge.  The CUDA path (red-black smoothing, FP64 and mixed)
is compared through the C ABI with the oracle, whose stiffness comes from element assembly
with the per-element coefficient (eq. 2.3):
  * single steps (residual, red-black sweeps, a V-cycle) at 1e-13 / 1e-12 relative;
  * the level-1 Newton solve, one correction step and the whole FMG solve at 1e-10 (FP64);
  * the mixed path within a tenth of the discretization error (estimated by Richardson from
    the exact discrete solutions on two levels: no closed form with a coefficient that jumps
    across the cells of T_H), and its algebraic error below a tenth of it.
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


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def problem(dim, H, r, f="cubic"):
    modes = [((1, 1), 3.0), ((2, 3), -1.5), ((4, 1), 1.0)] if dim == 2 else [((1, 1, 1), 3.0), ((2, 1, 3), -1.5)]
    return W.Problem(dim=dim, coarse_cells=H, refinements=r, f=f, a=1.0, g_modes=modes,
                     coefficient=W.cell_coefficient(dim, H))


def solver(F, prob, precision="fp64", **kw):
    return F.Solver(F.make_params(prob, precision=precision, **kw), prob.g_nodal())


# ---------------------------------------------------------------------------- single steps

@pytest.mark.parametrize("dim,H,r", [(2, 4, 3), (2, 8, 2), (3, 4, 2), (3, 2, 3)])
def test_residual_smoother_and_cycle_match_oracle(fmg, dim, H, r):
    prob = problem(dim, H, r)
    s = solver(fmg, prob)
    hier = O.build_hierarchy(dim, H, r, coef=prob.coefficient)
    rng = np.random.default_rng(5)
    for k in range(1, r + 2):
        lev = hier.level(k)
        u = rng.standard_normal(lev.A.shape[0])
        b = rng.standard_normal(lev.A.shape[0]) * lev.h ** dim
        rd = torch.zeros((lev.n + 1,) * dim, dtype=torch.float64, device="cuda")
        fmg.fmg_op_residual(s.ctx, k, dev(O.to_nodal(lev, b)), dev(O.to_nodal(lev, u)), rd)
        assert rel(O.from_nodal(lev, rd.cpu().numpy()), b - lev.A @ u) <= 1e-13, k
        for order in (0, 1):
            ud = dev(O.to_nodal(lev, u))
            fmg.fmg_op_smooth(s.ctx, k, dev(O.to_nodal(lev, b)), ud, 2, order)
            ref = u.copy()
            O.smooth(lev, b, ref, 2, ("red", "black") if order == 0 else ("black", "red"))
            assert rel(O.from_nodal(lev, ud.cpu().numpy()), ref) <= 1e-13, (k, order)
            u32 = dev(O.to_nodal(lev, u), torch.float32)
            fmg.fmg_op_smooth_f32(s.ctx, k, dev(O.to_nodal(lev, b), torch.float32), u32, 2, order)
            assert rel(O.from_nodal(lev, u32.double().cpu().numpy()), ref) <= 2e-5, (k, order)
    # two V-cycles on the finest level (per-level kernels down to the exact level-1 solve)
    k = r + 1
    lev = hier.level(k)
    b = rng.standard_normal(lev.A.shape[0]) * lev.h ** dim
    u = rng.standard_normal(lev.A.shape[0]) * 0.1
    ud = dev(O.to_nodal(lev, u))
    fmg.fmg_op_vcycle(s.ctx, k, dev(O.to_nodal(lev, b)), ud, 2)
    ref = O.vcycle(hier, k, b, O.vcycle(hier, k, b, u))
    assert rel(O.from_nodal(lev, ud.cpu().numpy()), ref) <= 1e-12
    s.close()


def test_coefficient_changes_the_operator(fmg):
    """The residual of a context with A(x) differs from A = I (the table is used), and A = 2 I
    doubles the A = I operator (to rounding: the weighted and the constant stencils sum in
    different orders)."""
    prob = problem(2, 4, 2)
    lev = O.assemble_level(2, 16)
    rng = np.random.default_rng(1)
    u = dev(O.to_nodal(lev, rng.standard_normal(lev.A.shape[0])))
    zero = torch.zeros_like(u)
    out = {}
    for name, coef in (("I", None), ("A", prob.coefficient), ("2I", np.full((16, 2), 2.0))):
        s = fmg.Solver(fmg.make_params(prob, coefficient=coef), prob.g_nodal())
        r = torch.zeros_like(u)
        fmg.fmg_op_residual(s.ctx, 3, zero, u, r)
        out[name] = r.cpu().numpy()
        s.close()
    assert np.max(np.abs(out["A"] - out["I"])) > 0.1 * np.max(np.abs(out["I"]))
    assert rel(out["2I"], 2.0 * out["I"]) <= 1e-14


@pytest.mark.parametrize("dim,H,f", [(2, 4, "cubic"), (2, 8, "expm1"), (3, 4, "expm1"), (3, 2, "cubic")])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_level1_solve_matches_oracle(fmg, dim, H, f, precision):
    prob = problem(dim, H, 2, f)
    s = solver(fmg, prob, precision)
    lev = O.assemble_level(dim, H, coef=prob.coefficient, coef_cells=H)
    G = O.load_vector(lev, O.restrict_nodal(prob.g_nodal(), dim, prob.n_fine, H))
    ref, its = O.newton_full(lev, G, f, prob.a, tol=1e-6, direct="dense")
    ud = torch.zeros((H + 1,) * dim, dtype=torch.float64, device="cuda")
    st = fmg.fmg_stats()
    fmg.fmg_op_level1_solve(s.ctx, ud, st)
    assert rel(O.from_nodal(lev, ud.cpu().numpy()), ref) <= FP64_TOL
    if precision == "fp64":
        assert abs(st.level1_iters - its) <= 1
    s.close()


@pytest.mark.parametrize("dim,H,r,f", [(2, 4, 3, "cubic"), (2, 8, 2, "expm1"), (3, 4, 2, "expm1"),
                                       (3, 2, 2, "cubic")])
def test_correction_step_matches_oracle(fmg, dim, H, r, f):
    prob = problem(dim, H, r, f)
    s = solver(fmg, prob)
    hier = O.build_hierarchy(dim, H, r, coef=prob.coefficient)
    k = r + 1
    lev = hier.level(k)
    G = O.load_vector(lev, prob.g_nodal())
    ub, _ = O.newton_full(lev, G, f, prob.a)
    u0 = ub + 0.05 * np.random.default_rng(9).standard_normal(ub.shape)
    ref, info = O.correction_step(hier, k, u0, G, f, prob.a)
    ud = dev(O.to_nodal(lev, u0))
    st = fmg.fmg_stats()
    fmg.fmg_op_correction_step(s.ctx, k, ud, st)
    assert rel(O.from_nodal(lev, ud.cpu().numpy()), ref) <= FP64_TOL
    assert abs(st.alpha[k - 1] - info.alpha) <= 1e-10
    assert abs(st.newton_iters[k - 1] - info.newton_iters) <= 1
    s.close()


# ---------------------------------------------------------------------------- full multigrid

FMG_CASES = [(2, 4, 4, "cubic"), (2, 8, 3, "expm1"), (2, 8, 5, "cubic"), (3, 4, 2, "expm1"), (3, 4, 3, "expm1"),
             (3, 2, 3, "cubic")]


def reference(prob, hier):
    """Oracle FMG, the exact discrete solution on the finest level and one level below, and the
    Richardson estimate of the discretization error ||u_bar_h - P u_bar_2h|| / 3."""
    dim, r = prob.dim, prob.refinements
    g = prob.g_nodal()
    res = O.fmg(hier, g, prob.f, prob.a, m=prob.m_vcycles)
    lev, levc = hier.level(r + 1), hier.level(r)
    ub, _ = O.newton_full(lev, O.load_vector(lev, g), prob.f, prob.a, U0=res.u[-1])
    ubc, _ = O.newton_full(levc, O.load_vector(levc, O.restrict_nodal(g, dim, prob.n_fine, levc.n)), prob.f,
                           prob.a, U0=res.u[-2])
    return res, ub, O.discrete_l2(lev, ub - lev.P @ ubc) / 3.0


@pytest.mark.parametrize("dim,H,r,f", FMG_CASES)
def test_fmg_matches_oracle(fmg, dim, H, r, f):
    prob = problem(dim, H, r, f)
    if dim == 3:
        prob.m_vcycles = W.M_VCYCLES_3D
    hier = O.build_hierarchy(dim, H, r, coef=prob.coefficient)
    res, ub, e_disc = reference(prob, hier)
    lev = hier.level(r + 1)
    # FP64 path, element by element
    s = solver(fmg, prob)
    st = fmg.fmg_stats()
    u64 = O.from_nodal(lev, s.solve(stats=st).cpu().numpy())
    s.close()
    assert st.flags == 0
    assert rel(u64, res.u[-1]) <= FP64_TOL
    for k, info in res.steps:
        assert abs(st.newton_iters[k - 1] - info.newton_iters) <= 1
        assert abs(st.alpha[k - 1] - info.alpha) <= 1e-9
    # Theorem 3.2's bar holds for the oracle's result (and so for the FP64 path)
    assert O.discrete_l2(lev, res.u[-1] - ub) <= 0.1 * e_disc
    # mixed path: within a tenth of the discretization error of the FP64 result and of u_bar
    s = solver(fmg, prob, "mixed")
    st = fmg.fmg_stats()
    umx = O.from_nodal(lev, s.solve(stats=st).cpu().numpy())
    s.close()
    assert st.flags == 0
    assert O.discrete_l2(lev, umx - res.u[-1]) <= 0.1 * e_disc
    assert O.discrete_l2(lev, umx - ub) <= 0.1 * e_disc


def test_fmg_with_coefficient_at_the_benchmark_shape(fmg):
    """2D H = 1/8 at 7 refinements (1025^2 nodes: the augmented kernel with several blocks per
    coarse cell and the float-float level start): FP64 against the oracle at 1e-10, mixed at the
    discretization bar."""
    prob = W.config_coefficient(2, refinements=7)
    hier = O.build_hierarchy(2, 8, 7, coef=prob.coefficient)
    res, ub, e_disc = reference(prob, hier)
    lev = hier.level(8)
    for precision in ("fp64", "mixed"):
        s = solver(fmg, prob, precision)
        st = fmg.fmg_stats()
        u = O.from_nodal(lev, s.solve(stats=st).cpu().numpy())
        s.close()
        assert st.flags == 0, precision
        if precision == "fp64":
            assert rel(u, res.u[-1]) <= FP64_TOL
        assert O.discrete_l2(lev, u - ub) <= 0.1 * e_disc, precision


def test_batches_and_server_reject_a_coefficient(fmg):
    prob = problem(2, 4, 2)
    s = solver(fmg, prob)
    with pytest.raises(fmg.FMGError) as ei:
        fmg.Batch([s])
    assert ei.value.status == fmg.FMG_ERR_INVALID
    s.close()

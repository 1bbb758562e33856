"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 path: element-wise agreement within 1e-10 relative in the max norm (the
FP64 bar; reductions run in a different order, so bit equality is not
expected).  Mixed path: difference to the oracle's FP64 result below a tenth
of the discretization error.  Single-kernel steps (smoother, residual,
prolongation) are held to 1e-13 relative.
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


def make_solver(F, prob, precision="fp64", **kw):
    return F.Solver(F.make_params(prob, precision=precision, **kw), prob.g_nodal())


def prob2d(H=4, r=3, f="cubic", a=1.0):
    return W.Problem(dim=2, coarse_cells=H, refinements=r, f=f, a=a,
                     modes=[((1, 1), 1.0), ((2, 3), 0.5), ((5, 1), -0.3)])


def prob3d(H=4, r=2, f="expm1", a=1.0):
    return W.Problem(dim=3, coarse_cells=H, refinements=r, f=f, a=a,
                     modes=[((1, 1, 1), 0.8), ((2, 1, 3), 0.4)])


# ---------------------------------------------------------------------------- single steps

@pytest.mark.parametrize("dim,H,r,level", [(2, 4, 3, 4), (2, 8, 2, 3), (3, 4, 2, 3), (3, 4, 1, 2)])
@pytest.mark.parametrize("order", [0, 1])
def test_rbgs_matches_oracle(fmg, dim, H, r, level, order):
    prob = prob2d(H, r) if dim == 2 else prob3d(H, r)
    s = make_solver(fmg, prob)
    lev = O.assemble_level(dim, H << (level - 1))
    rng = np.random.default_rng(11)
    u0 = rng.standard_normal(lev.A.shape[0])
    b = rng.standard_normal(lev.A.shape[0]) * lev.h ** dim
    ud = dev(O.to_nodal(lev, u0))
    bd = dev(O.to_nodal(lev, b))
    fmg.fmg_op_smooth(s.ctx, level, bd, ud, 3, order)
    ref = u0.copy()
    O.smooth(lev, b, ref, 3, ("red", "black") if order == 0 else ("black", "red"))
    got = O.from_nodal(lev, ud.cpu().numpy())
    assert rel(got, ref) <= 1e-13
    # boundary untouched (zero)
    full = ud.cpu().numpy().ravel()
    mask = np.ones(full.size, bool)
    mask[lev.interior] = False
    assert np.all(full[mask] == 0.0)
    # FP32 smoother on the same data
    u32 = dev(O.to_nodal(lev, u0), torch.float32)
    b32 = dev(O.to_nodal(lev, b), torch.float32)
    fmg.fmg_op_smooth_f32(s.ctx, level, b32, u32, 3, order)
    got32 = O.from_nodal(lev, u32.double().cpu().numpy())
    assert rel(got32, ref) <= 2e-5
    s.close()


@pytest.mark.parametrize("dim,H,r", [(2, 4, 3), (3, 4, 2)])
def test_residual_and_prolongation_match_oracle(fmg, dim, H, r):
    prob = prob2d(H, r) if dim == 2 else prob3d(H, r)
    s = make_solver(fmg, prob)
    hier = O.build_hierarchy(dim, H, r)
    rng = np.random.default_rng(5)
    for k in range(2, r + 2):
        lev = hier.level(k)
        u = rng.standard_normal(lev.A.shape[0])
        b = rng.standard_normal(lev.A.shape[0])
        rd = torch.zeros((lev.n + 1,) * dim, dtype=torch.float64, device="cuda")
        fmg.fmg_op_residual(s.ctx, k, dev(O.to_nodal(lev, b)), dev(O.to_nodal(lev, u)), rd)
        ref = b - lev.A @ u
        assert rel(O.from_nodal(lev, rd.cpu().numpy()), ref) <= 1e-13
        coarse = hier.level(k - 1)
        ec = rng.standard_normal(coarse.A.shape[0])
        uf = torch.full((lev.n + 1,) * dim, 7.0, dtype=torch.float64, device="cuda")
        fmg.fmg_op_prolong(s.ctx, k, dev(O.to_nodal(coarse, ec)), uf)
        assert rel(O.from_nodal(lev, uf.cpu().numpy()), lev.P @ ec) <= 1e-15
    s.close()


@pytest.mark.parametrize("dim,H,r", [(2, 4, 4), (2, 8, 3), (3, 4, 3)])
def test_vcycle_matches_oracle(fmg, dim, H, r):
    prob = prob2d(H, r) if dim == 2 else prob3d(H, r)
    s = make_solver(fmg, prob)
    hier = O.build_hierarchy(dim, H, r)
    k = r + 1
    lev = hier.level(k)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(lev.A.shape[0]) * lev.h ** dim
    u = rng.standard_normal(lev.A.shape[0]) * 0.1
    ud = dev(O.to_nodal(lev, u))
    fmg.fmg_op_vcycle(s.ctx, k, dev(O.to_nodal(lev, b)), ud, 2)
    ref = O.vcycle(hier, k, b, O.vcycle(hier, k, b, u))
    assert rel(O.from_nodal(lev, ud.cpu().numpy()), ref) <= 1e-12
    s.close()


def test_mixed_vcycle_contracts_like_fp64(fmg):
    """Defect correction: FP32 cycle inside FP64 residual/update keeps the FP64 V-cycle's
    contraction until the FP64 solution is reached to ~1e-12."""
    prob = prob2d(4, 5)
    s = make_solver(fmg, prob, precision="mixed")
    hier = O.build_hierarchy(2, 4, 5)
    k = 6
    lev = hier.level(k)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(lev.A.shape[0]) * lev.h ** 2
    import scipy.sparse.linalg as spla

    x = spla.spsolve(lev.A.tocsc(), b)
    ud = torch.zeros((lev.n + 1,) * 2, dtype=torch.float64, device="cuda")
    bd = dev(O.to_nodal(lev, b))
    errs = []
    for _ in range(30):
        fmg.fmg_op_vcycle(s.ctx, k, bd, ud, 1)
        errs.append(np.max(np.abs(O.from_nodal(lev, ud.cpu().numpy()) - x)))
    assert errs[3] / errs[0] < 0.25 ** 3
    assert errs[-1] <= 1e-12 * np.max(np.abs(x))
    s.close()


@pytest.mark.parametrize("dim,H,kind", [(2, 4, "cubic"), (2, 8, "expm1"), (3, 4, "expm1"), (2, 4, "neg_exp_neg")])
def test_level1_solve_matches_oracle(fmg, dim, H, kind):
    prob = prob2d(H, 2, kind) if dim == 2 else prob3d(H, 1, kind)
    s = make_solver(fmg, prob)
    g = prob.g_nodal()
    lev = O.assemble_level(dim, H)
    G = O.load_vector(lev, O.restrict_nodal(g, dim, prob.n_fine, H))
    ref, its = O.newton_full(lev, G, kind, prob.a, tol=1e-6, direct="dense")
    ud = torch.zeros((H + 1,) * dim, dtype=torch.float64, device="cuda")
    st = fmg.fmg_stats()
    fmg.fmg_op_level1_solve(s.ctx, ud, st)
    assert rel(O.from_nodal(lev, ud.cpu().numpy()), ref) <= FP64_TOL
    assert abs(st.level1_iters - its) <= 1
    s.close()


@pytest.mark.parametrize("dim,H,r,kind", [(2, 4, 3, "cubic"), (2, 8, 2, "expm1"), (3, 4, 2, "expm1"),
                                          (2, 4, 4, "signed_pow32"), (3, 4, 1, "cubic")])
def test_correction_step_matches_oracle(fmg, dim, H, r, kind):
    prob = prob2d(H, r, kind) if dim == 2 else prob3d(H, r, kind)
    s = make_solver(fmg, prob)
    hier = O.build_hierarchy(dim, H, r)
    k = r + 1
    lev = hier.level(k)
    G = O.load_vector(lev, prob.g_nodal())
    rng = np.random.default_rng(9)
    ub, _ = O.newton_full(lev, G, kind, prob.a)
    u0 = ub + 0.05 * rng.standard_normal(ub.shape)
    ref, info = O.correction_step(hier, k, u0, G, kind, prob.a)
    ud = dev(O.to_nodal(lev, u0))
    st = fmg.fmg_stats()
    fmg.fmg_op_correction_step(s.ctx, k, ud, st)
    assert rel(O.from_nodal(lev, ud.cpu().numpy()), ref) <= FP64_TOL
    assert abs(st.alpha[k - 1] - info.alpha) <= 1e-10
    assert abs(st.newton_iters[k - 1] - info.newton_iters) <= 1
    s.close()


# ---------------------------------------------------------------------------- full multigrid

FMG_CASES = [
    (2, 4, 4, "cubic"), (2, 4, 5, "expm1"), (2, 8, 3, "cubic"), (2, 4, 4, "signed_pow32"),
    (2, 4, 4, "neg_exp_neg"), (2, 4, 3, "linear"), (3, 4, 2, "expm1"), (3, 4, 3, "cubic"),
    (2, 2, 3, "cubic"), (3, 2, 2, "cubic"),
]


@pytest.mark.parametrize("dim,H,r,kind", FMG_CASES)
def test_fmg_fp64_matches_oracle(fmg, dim, H, r, kind):
    prob = prob2d(H, r, kind) if dim == 2 else prob3d(H, r, kind)
    hier = O.build_hierarchy(dim, H, r)
    res = O.fmg(hier, prob.g_nodal(), kind, prob.a)
    s = make_solver(fmg, prob)
    st = fmg.fmg_stats()
    u = s.solve(stats=st).cpu().numpy()
    ref = O.to_nodal(hier.level(r + 1), res.u[-1])
    assert rel(u, ref) <= FP64_TOL
    assert st.level1_iters == res.level1_iters or abs(st.level1_iters - res.level1_iters) <= 1
    for k, info in res.steps:
        assert abs(st.newton_iters[k - 1] - info.newton_iters) <= 1
        assert abs(st.alpha[k - 1] - info.alpha) <= 1e-9
    assert st.flags == 0
    s.close()


@pytest.mark.parametrize("dim,H,r,kind", [(2, 4, 5, "cubic"), (2, 8, 4, "expm1"), (3, 4, 3, "expm1")])
def test_fmg_mixed_below_discretization_error(fmg, dim, H, r, kind):
    prob = prob2d(H, r, kind) if dim == 2 else prob3d(H, r, kind)
    hier = O.build_hierarchy(dim, H, r)
    g = prob.g_nodal()
    res = O.fmg(hier, g, kind, prob.a)
    lev = hier.level(r + 1)
    ub, _ = O.newton_full(lev, O.load_vector(lev, g), kind, prob.a, U0=res.u[-1])
    e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star()))
    s = make_solver(fmg, prob, precision="mixed")
    u = O.from_nodal(lev, s.solve().cpu().numpy())
    # the mixed result stays within a tenth of the discretization error of the FP64 method
    assert O.discrete_l2(lev, u - res.u[-1]) <= 0.1 * e_disc
    # and its algebraic error is that of the FP64 method up to the same margin
    e_alg64 = O.discrete_l2(lev, res.u[-1] - ub)
    assert O.discrete_l2(lev, u - ub) <= e_alg64 + 0.1 * e_disc
    s.close()


def test_solve_is_deterministic_and_repeatable(fmg):
    prob = prob2d(8, 4, "cubic")
    s = make_solver(fmg, prob)
    a = s.solve().cpu().numpy()
    b = s.solve().cpu().numpy()
    assert np.array_equal(a, b)
    s2 = make_solver(fmg, prob)
    c = s2.solve().cpu().numpy()
    assert np.array_equal(a, c)
    s.close()
    s2.close()


def test_set_rhs_and_host_io(fmg):
    p1 = prob2d(4, 4, "cubic")
    p2 = W.Problem(dim=2, coarse_cells=4, refinements=4, f="cubic", modes=[((2, 2), -1.0)])
    s = make_solver(fmg, p1)
    params = fmg.make_params(p2)
    ref2 = O.fmg(O.build_hierarchy(2, 4, 4), p2.g_nodal(), "cubic", 1.0)
    s.set_rhs(p2.g_nodal())
    host = np.zeros((65, 65))
    fmg.fmg_solve(s.ctx, host)
    assert rel(host, O.to_nodal(O.assemble_level(2, 64), ref2.u[-1])) <= FP64_TOL
    del params
    s.close()


def test_refinements_zero_is_the_level1_solve(fmg):
    prob = W.Problem(dim=2, coarse_cells=8, refinements=0, f="cubic", modes=[((1, 1), 1.0)])
    s = make_solver(fmg, prob)
    u = s.solve().cpu().numpy()
    lev = O.assemble_level(2, 8)
    ref, _ = O.newton_full(lev, O.load_vector(lev, prob.g_nodal()), "cubic", 1.0, tol=1e-6, direct="dense")
    assert rel(u, O.to_nodal(lev, ref)) <= 1e-10
    s.close()


def test_zero_rhs_gives_zero_and_flags_dropped_basis(fmg):
    prob = W.Problem(dim=2, coarse_cells=4, refinements=3, f="cubic", g_const=0.0)
    s = make_solver(fmg, prob)
    st = fmg.fmg_stats()
    u = s.solve(stats=st).cpu().numpy()
    assert np.all(u == 0.0)
    assert st.flags & 4
    s.close()


def test_errors_are_reported(fmg):
    prob = prob2d(4, 3, "cubic")
    g = prob.g_nodal()
    g_bad = g.copy()
    g_bad[10, 10] = np.nan
    s = fmg.Solver(fmg.make_params(prob), g_bad)
    with pytest.raises(fmg.FMGError) as ei:
        s.solve(stats=fmg.fmg_stats())
    assert ei.value.status in (fmg.FMG_ERR_NONFINITE, fmg.FMG_ERR_NO_CONVERGENCE)
    s.close()
    s = fmg.Solver(fmg.make_params(prob, newton_maxit=1, newton_tol=1e-300), g)
    with pytest.raises(fmg.FMGError) as ei:
        s.solve(stats=fmg.fmg_stats())
    assert ei.value.status == fmg.FMG_ERR_NO_CONVERGENCE
    s.close()
    # the context stays usable after an error report
    s = fmg.Solver(fmg.make_params(prob), g)
    s.solve(stats=fmg.fmg_stats())
    s.close()


@pytest.mark.parametrize("dim,H,r,nu", [(2, 4, 6, 2), (2, 8, 4, 1), (2, 4, 5, 3), (3, 4, 3, 2)])
def test_mixed_cycle_equals_fp64_cycle_to_fp32_precision(fmg, dim, H, r, nu):
    """One mixed-precision cycle (fused FP32 kernels in 2D for nu <= 2, per-step kernels
    otherwise) moves u by the FP64 cycle's correction up to FP32 rounding."""
    prob = prob2d(H, r) if dim == 2 else prob3d(H, r)
    prob.nu_pre = prob.nu_post = nu
    s = make_solver(fmg, prob, precision="mixed")
    hier = O.build_hierarchy(dim, H, r)
    k = r + 1
    lev = hier.level(k)
    rng = np.random.default_rng(8)
    b = rng.standard_normal(lev.A.shape[0]) * lev.h ** dim
    u = 0.3 * rng.standard_normal(lev.A.shape[0])
    ud = dev(O.to_nodal(lev, u))
    fmg.fmg_op_vcycle(s.ctx, k, dev(O.to_nodal(lev, b)), ud, 1)
    ref = O.vcycle(hier, k, b, u, nu, nu)
    got = O.from_nodal(lev, ud.cpu().numpy())
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref - u))
    s.close()


@pytest.mark.parametrize("dim,H,r,kind,p", [(2, 4, 4, "cubic", 2), (3, 4, 2, "expm1", 3)])
def test_fmg_several_correction_steps_per_level(fmg, dim, H, r, kind, p):
    """Algorithm 3.2 with p > 1 correction steps per level: every level's steps repeat
    Algorithm 3.1 from the previous step's result."""
    prob = prob2d(H, r, kind) if dim == 2 else prob3d(H, r, kind)
    hier = O.build_hierarchy(dim, H, r)
    res = O.fmg(hier, prob.g_nodal(), kind, prob.a, p=p)
    s = make_solver(fmg, prob, p_corrections=p)
    st = fmg.fmg_stats()
    u = s.solve(stats=st).cpu().numpy()
    assert st.flags == 0
    assert rel(u, O.to_nodal(hier.level(r + 1), res.u[-1])) <= FP64_TOL
    # the per-level Newton counts are summed over the p steps
    for k in range(2, r + 2):
        want = sum(info.newton_iters for kk, info in res.steps if kk == k)
        assert abs(st.newton_iters[k - 1] - want) <= p
    s.close()


@pytest.mark.parametrize("dim,H,r,kind", [(2, 4, 4, "cubic"), (2, 8, 3, "cubic"), (3, 4, 2, "cubic"),
                                          (2, 4, 4, "expm1")])
def test_fmg_fixed_point_fp64_matches_oracle(fmg, dim, H, r, kind):
    """The fixed-point variant of the augmented solve (Galerkin stiffness factored once)."""
    prob = prob2d(H, r, kind) if dim == 2 else prob3d(H, r, kind)
    hier = O.build_hierarchy(dim, H, r)
    res = O.fmg(hier, prob.g_nodal(), kind, prob.a, nonlinear="fixed_point")
    s = make_solver(fmg, prob, nonlinear="fixed_point", newton_maxit=60)
    st = fmg.fmg_stats()
    u = s.solve(stats=st).cpu().numpy()
    assert st.flags == 0
    assert rel(u, O.to_nodal(hier.level(r + 1), res.u[-1])) <= FP64_TOL
    for k, info in res.steps:
        assert abs(st.newton_iters[k - 1] - info.newton_iters) <= 1
    s.close()


@pytest.mark.parametrize("dim,H,r,kind", [(2, 4, 5, "cubic"), (3, 4, 3, "cubic")])
def test_fmg_fixed_point_mixed_below_discretization_error(fmg, dim, H, r, kind):
    prob = prob2d(H, r, kind) if dim == 2 else prob3d(H, r, kind)
    hier = O.build_hierarchy(dim, H, r)
    g = prob.g_nodal()
    res = O.fmg(hier, g, kind, prob.a, nonlinear="fixed_point")
    lev = hier.level(r + 1)
    ub, _ = O.newton_full(lev, O.load_vector(lev, g), kind, prob.a, U0=res.u[-1])
    e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star()))
    s = make_solver(fmg, prob, precision="mixed", nonlinear="fixed_point", newton_maxit=60)
    st = fmg.fmg_stats()
    u = O.from_nodal(lev, s.solve(stats=st).cpu().numpy())
    assert st.flags == 0
    assert O.discrete_l2(lev, u - res.u[-1]) <= 0.1 * e_disc
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_paper_examples_2_and_3_on_the_cube(fmg, precision):
    """Sec. 4's second and third examples on the unit cube: f = -exp(-u) with g = 1 (no
    manufactured solution), and the odd extension of u^{3/2} with u* = prod sin(2 pi x_i)."""
    ex2 = W.Problem(dim=3, coarse_cells=4, refinements=2, f="neg_exp_neg", a=1.0, g_const=1.0)
    ex3 = W.Problem(dim=3, coarse_cells=4, refinements=2, f="signed_pow32", a=1.0, modes=[((2, 2, 2), 1.0)])
    for prob in (ex2, ex3):
        hier = O.build_hierarchy(3, 4, 2)
        g = prob.g_nodal()
        res = O.fmg(hier, g, prob.f, prob.a)
        lev = hier.level(3)
        s = make_solver(fmg, prob, precision=precision)
        st = fmg.fmg_stats()
        u = s.solve(stats=st).cpu().numpy()
        assert st.flags == 0
        if precision == "fp64":
            assert rel(u, O.to_nodal(lev, res.u[-1])) <= FP64_TOL
        else:
            # against the exact discrete solution: the mixed result's algebraic error is the
            # FP64 method's up to FP32-level rounding
            ub, _ = O.newton_full(lev, O.load_vector(lev, g), prob.f, prob.a, U0=res.u[-1])
            e_alg64 = O.discrete_l2(lev, res.u[-1] - ub)
            e_mixed = O.discrete_l2(lev, O.from_nodal(lev, u) - ub)
            assert e_mixed <= e_alg64 + 1e-6 * O.discrete_l2(lev, ub)
        s.close()

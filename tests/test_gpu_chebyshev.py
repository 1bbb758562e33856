"""Chebyshev-Jacobi smoothing on the GPU (through the C ABI) against the FP64 oracle.

Each Chebyshev step is one colour-free stencil pass; the FP64 path is held to the FP64 bar
(1e-13 relative for single steps and cycles, 1e-10 for whole FMG solves), the FP32 steps and
the mixed path to their FP32 and discretization bars.
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


def problem(dim, H, r, f="cubic", m=2):
    modes = [((1,) * dim, 1.0), ((2, 1, 3)[:dim], 0.5)]
    return W.Problem(dim=dim, coarse_cells=H, refinements=r, f=f, a=1.0, modes=modes, m_vcycles=m)


def solver(F, prob, precision):
    return F.Solver(F.make_params(prob, precision=precision, smoother="chebyshev"), prob.g_nodal())


@pytest.mark.parametrize("dim,H,r,level", [(2, 4, 3, 4), (2, 8, 2, 3), (3, 4, 2, 3)])
@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_chebyshev_steps_match_oracle(fmg, dim, H, r, level, degree):
    s = solver(fmg, problem(dim, H, r), "mixed")
    lev = O.assemble_level(dim, H << (level - 1))
    rng = np.random.default_rng(17)
    u0 = rng.standard_normal(lev.A.shape[0])
    b = rng.standard_normal(lev.A.shape[0]) * lev.h ** dim
    ud = dev(O.to_nodal(lev, u0))
    fmg.fmg_op_smooth(s.ctx, level, dev(O.to_nodal(lev, b)), ud, degree, 0)
    ref = u0.copy()
    O.chebyshev_smooth(lev, b, ref, degree)
    assert rel(O.from_nodal(lev, ud.cpu().numpy()), ref) <= 1e-13
    full = ud.cpu().numpy().ravel()
    mask = np.ones(full.size, bool)
    mask[lev.interior] = False
    assert np.all(full[mask] == 0.0)
    u32 = dev(O.to_nodal(lev, u0), torch.float32)
    fmg.fmg_op_smooth_f32(s.ctx, level, dev(O.to_nodal(lev, b), torch.float32), u32, degree, 0)
    assert rel(O.from_nodal(lev, u32.double().cpu().numpy()), ref) <= 2e-5
    s.close()


@pytest.mark.parametrize("dim,H,r", [(2, 4, 4), (2, 8, 3), (3, 4, 3)])
def test_chebyshev_vcycle_matches_oracle(fmg, dim, H, r):
    """Covers the per-level Chebyshev kernel and the Chebyshev steps of the one-CTA coarse
    cycle (levels up to 64^2 / 16^3)."""
    s = solver(fmg, problem(dim, H, r), "fp64")
    hier = O.build_hierarchy(dim, H, r)
    k = r + 1
    lev = hier.level(k)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(lev.A.shape[0]) * lev.h ** dim
    u = rng.standard_normal(lev.A.shape[0]) * 0.1
    ud = dev(O.to_nodal(lev, u))
    fmg.fmg_op_vcycle(s.ctx, k, dev(O.to_nodal(lev, b)), ud, 2)
    ref = O.vcycle(hier, k, b, O.vcycle(hier, k, b, u, smoother="chebyshev"), smoother="chebyshev")
    assert rel(O.from_nodal(lev, ud.cpu().numpy()), ref) <= 1e-12
    s.close()


@pytest.mark.parametrize("dim,H,r,f,m", [(2, 4, 4, "cubic", 2), (2, 8, 3, "expm1", 2), (3, 4, 2, "expm1", 3),
                                         (2, 4, 5, "neg_exp_neg", 2)])
def test_fmg_chebyshev_fp64_matches_oracle(fmg, dim, H, r, f, m):
    prob = problem(dim, H, r, f, m)
    hier = O.build_hierarchy(dim, H, r)
    res = O.fmg(hier, prob.g_nodal(), f, prob.a, m=m, smoother="chebyshev")
    s = solver(fmg, prob, "fp64")
    st = fmg.fmg_stats()
    u = s.solve(stats=st).cpu().numpy()
    assert st.flags == 0
    assert rel(u, O.to_nodal(hier.level(r + 1), res.u[-1])) <= FP64_TOL
    for k, info in res.steps:
        assert abs(st.newton_iters[k - 1] - info.newton_iters) <= 1
    s.close()


@pytest.mark.parametrize("dim,H,r,f,m", [(2, 4, 5, "cubic", 2), (2, 8, 4, "expm1", 2), (3, 4, 3, "expm1", 3)])
def test_fmg_chebyshev_mixed_below_discretization_error(fmg, dim, H, r, f, m):
    prob = problem(dim, H, r, f, m)
    hier = O.build_hierarchy(dim, H, r)
    g = prob.g_nodal()
    res = O.fmg(hier, g, f, prob.a, m=m, smoother="chebyshev")
    lev = hier.level(r + 1)
    ub, _ = O.newton_full(lev, O.load_vector(lev, g), f, prob.a, U0=res.u[-1])
    e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star()))
    s = solver(fmg, prob, "mixed")
    u = O.from_nodal(lev, s.solve().cpu().numpy())
    assert O.discrete_l2(lev, u - res.u[-1]) <= 0.1 * e_disc
    e_alg64 = O.discrete_l2(lev, res.u[-1] - ub)
    assert O.discrete_l2(lev, u - ub) <= e_alg64 + 0.1 * e_disc
    s.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autotuned_shapes_give_the_same_bits(fmg, precision):
    """The autotuner only changes how nodes are dealt to threads: every node is computed the
    same way, so the solve gives the same bits before and after tuning."""
    prob = problem(2, 4, 6, "cubic")
    s = solver(fmg, prob, precision)
    before = s.solve().cpu().numpy()
    tuned = fmg.fmg_autotune(s.ctx)
    assert tuned >= 1
    for level in range(1, prob.levels + 1):
        block, strip = fmg.fmg_tuned_shape(s.ctx, level)
        assert block in (64, 128, 256, 512) and strip in (1, 2, 4, 8)
    after = s.solve().cpu().numpy()
    assert np.array_equal(before, after)
    s.close()

"""The augmented Newton kernel's launch-shape autotuner (fmg_autotune_augmented) against the
FP64 oracle.

The tuned shape (column-chunk length, blocks per coarse cell) changes only how the fine pass is
dealt to threads and so the order of the block sums: a tuned context still solves to the FP64
bar (1e-10 relative against the oracle) and to the mixed path's bar, and two of its solves give
the same bits.  The tuned shapes are process-wide, so this file runs after the other GPU tests
(which assume the default rule for bitwise comparisons of their own)."""
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


@pytest.mark.parametrize("dim,H,r", [(2, 4, 5), (2, 8, 4), (3, 4, 3)])
def test_tuned_augmented_shapes_keep_parity(fmg, dim, H, r):
    modes = [((1,) * dim, 1.0), ((2,) + (1,) * (dim - 1), 0.3)]
    prob = W.Problem(dim=dim, coarse_cells=H, refinements=r, f="cubic", modes=modes,
                     m_vcycles=2 if dim == 2 else 3)
    g = prob.g_nodal()
    hier = O.build_hierarchy(dim, H, r)
    lev = hier.level(r + 1)
    ref = O.fmg(hier, g, prob.f, prob.a, m=prob.m_vcycles, keep_levels=False).u[-1]
    ub, _ = O.newton_full(lev, O.load_vector(lev, g), prob.f, prob.a, U0=ref)
    e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star()))
    for prec in ("fp64", "mixed"):
        s = fmg.Solver(fmg.make_params(prob, precision=prec), g)
        assert fmg.fmg_autotune_augmented(s.ctx) == r
        for k in range(2, r + 2):
            chunk, bpc = fmg.fmg_aug_shape(s.ctx, k)
            assert 2 <= chunk <= 32 and chunk & (chunk - 1) == 0 and chunk <= max(2, 1 << (k - 1)), (k, chunk)
            assert bpc >= 1, (k, bpc)
        st = fmg.fmg_stats()
        u1 = s.solve(stats=st).cpu().numpy()
        assert st.flags == 0, prec
        u2 = s.solve().cpu().numpy()
        assert np.array_equal(u1, u2), prec
        u = O.from_nodal(lev, u1)
        if prec == "fp64":
            assert rel(u, ref) <= FP64_TOL
        else:
            assert O.discrete_l2(lev, u - ref) <= 0.1 * e_disc
        s.close()

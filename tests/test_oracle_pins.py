"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: textbook
stencils and weights (tests/golden/p1_stencils.txt), closed-form discrete
solutions, a brute-force sequential Gauss-Seidel, an independent root finder
and minimiser, invariances the method must have, and the convergence orders
and contraction properties stated in Sec. 2-3 (Lemma 2.1, eq. 3.5,
Theorem 3.1, Theorem 3.2, Corollary 3.1).
"""
import math
import os

import numpy as np
import pytest
import scipy.optimize as opt
import scipy.sparse as sp

from oracle import fmg_oracle as O
from paper_1611_05677_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "p1_stencils.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, dim, val = line.split()
        out[(key, int(dim))] = float(val)
    return out


# ---------------------------------------------------------------------------
# Discretization (Sec. 2, eq. 2.3 and 2.6; Sec. 3, eq. 3.1-3.3)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("dim,n", [(2, 4), (2, 16), (3, 4), (3, 8)])
def test_stiffness_is_textbook_stencil(dim, n):
    gd = golden()
    lev = O.assemble_level(dim, n)
    scale = lev.h ** (dim - 2)
    np.testing.assert_allclose(lev.A.diagonal() / scale, gd[("stiffness_diag_over_h^(d-2)", dim)], rtol=1e-13)
    # every off-diagonal entry is an axis neighbour with the textbook value
    A = lev.A.tocoo()
    off = A.row != A.col
    np.testing.assert_allclose(A.data[off] / scale, gd[("stiffness_axis_over_h^(d-2)", dim)], rtol=1e-13)
    nodes = lev.nodes[lev.interior]
    dist = np.abs(nodes[A.row[off]] - nodes[A.col[off]]).sum(axis=1)
    assert np.all(dist == 1)
    # and every interior axis neighbour pair is present
    assert off.sum() == sum(int(np.prod([n - 1] * (dim - 1))) * (n - 2) * 2 for _ in range(dim))


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_lumped_weights(dim, n):
    gd = golden()
    lev = O.assemble_level(dim, n)
    np.testing.assert_allclose(lev.w / lev.h ** dim, gd[("lumped_weight_over_h^d", dim)], rtol=1e-13)


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_energy_of_linear_function(dim, n):
    """a(l, l) = |grad l|^2 |Omega| for a linear l; the assembled matrix on all
    nodes must reproduce it exactly and annihilate constants."""
    lev = O.assemble_level(dim, n)
    X = lev.nodes * lev.h
    c = np.array([0.7, -1.3, 0.4][:dim])
    ell = X @ c + 0.25
    assert abs(ell @ (lev.S @ ell) - c @ c) < 1e-12
    assert np.max(np.abs(lev.S @ np.ones(lev.S.shape[0]))) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_is_refined_hat(dim):
    """Column of P for an interior coarse node = its hat on the refined mesh:
    1 at the node, 1/2 at the midpoints of the coarse edges leaving it."""
    gd = golden()
    nc = 4
    P = O.prolongation(dim, nc).tocsc()
    cnodes, _, _ = O.structured_mesh(dim, nc)
    fnodes, _, _ = O.structured_mesh(dim, 2 * nc)
    cin = cnodes[O.interior_mask(cnodes, nc)]
    fin = fnodes[O.interior_mask(fnodes, 2 * nc)]
    for col in range(P.shape[1]):
        z = 2 * cin[col]
        rows = P.indices[P.indptr[col]:P.indptr[col + 1]]
        vals = P.data[P.indptr[col]:P.indptr[col + 1]]
        offs = fin[rows] - z
        centre = np.all(offs == 0, axis=1)
        assert centre.sum() == 1 and vals[centre][0] == gd[("hat_refined_centre", dim)]
        edge = ~centre
        assert edge.sum() == gd[("hat_refined_edge_count", dim)]
        np.testing.assert_array_equal(vals[edge], gd[("hat_refined_edge_midpoint", dim)])
        # edge directions of the Freudenthal/Kuhn mesh: +-(0/1 vectors), all one sign
        o = offs[edge]
        assert np.all((np.all(o >= 0, axis=1)) | (np.all(o <= 0, axis=1)))
        assert np.all(np.abs(o) <= 1)


@pytest.mark.parametrize("dim,nc", [(2, 4), (2, 8), (3, 4)])
def test_galerkin_identity(dim, nc):
    """Nested P1 spaces: the coarse stiffness is the Galerkin product P^T A_h P."""
    Ac = O.assemble_level(dim, nc).A
    Af = O.assemble_level(dim, 2 * nc).A
    P = O.prolongation(dim, nc)
    assert abs(P.T @ Af @ P - Ac).max() < 1e-13


# ---------------------------------------------------------------------------
# Nonlinearities (Sec. 4) and Assumption A
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("kind", W.NONLINEARITIES)
def test_nonlinearity_derivatives_and_monotonicity(kind):
    u = np.linspace(-2.0, 2.0, 400)     # avoids u = 0, where |u|^{1/2} has no finite difference limit
    a = 1.7
    eps = 1e-6
    fd = (O.f_val(kind, a, u + eps) - O.f_val(kind, a, u - eps)) / (2 * eps)
    np.testing.assert_allclose(O.f_der(kind, a, u), fd, rtol=1e-6, atol=2e-6)
    pd = (O.f_antider(kind, a, u + eps) - O.f_antider(kind, a, u - eps)) / (2 * eps)
    np.testing.assert_allclose(pd, O.f_val(kind, a, u), rtol=1e-6, atol=1e-6)
    assert np.all(np.diff(O.f_val(kind, a, u)) >= 0)       # Assumption A, first condition


def test_nonlinearity_values():
    assert O.f_val("cubic", 2.0, np.array([1.5]))[0] == 6.75
    assert O.f_val("expm1", 1.0, np.array([0.0]))[0] == 0.0
    assert abs(O.f_val("expm1", 1.0, np.array([1.0]))[0] - (math.e - 1)) < 1e-15
    assert O.f_val("signed_pow32", 1.0, np.array([-4.0]))[0] == -8.0
    assert O.f_val("neg_exp_neg", 1.0, np.array([0.0]))[0] == -1.0


# ---------------------------------------------------------------------------
# Smoother and V-cycle (Algorithm 3.1 step 1, eq. 3.5)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_rbgs_equals_sequential_gauss_seidel(dim, n):
    """The vectorised colour update equals point Gauss-Seidel visiting all red
    unknowns, then all black ones, one at a time with a dense matrix."""
    lev = O.assemble_level(dim, n)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(lev.A.shape[0])
    u0 = rng.standard_normal(lev.A.shape[0])
    A = lev.A.toarray()
    us = u0.copy()
    for i in list(lev.red) + list(lev.black):
        us[i] = (b[i] - A[i] @ us + A[i, i] * us[i]) / A[i, i]
    uv = u0.copy()
    O.rbgs_half(lev, b, uv, "red")
    O.rbgs_half(lev, b, uv, "black")
    np.testing.assert_allclose(uv, us, rtol=0, atol=1e-13)
    assert O.same_colour_coupling(lev) == 0.0


@pytest.mark.parametrize("dim,H,r", [(2, 4, 3), (3, 4, 2)])
def test_vcycle_converges_to_direct_solution(dim, H, r):
    hier = O.build_hierarchy(dim, H, r)
    k = r + 1
    lev = hier.level(k)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(lev.A.shape[0]) * lev.h ** dim
    x = sp.linalg.spsolve(lev.A.tocsc(), b)
    u = np.zeros_like(b)
    for _ in range(30):
        u = O.vcycle(hier, k, b, u)
    assert np.max(np.abs(u - x)) <= 1e-12 * np.max(np.abs(x))


@pytest.mark.parametrize("dim,H,r,lo", [(2, 4, 5, 4), (3, 4, 4, 4)])
def test_vcycle_contraction_is_mesh_independent(dim, H, r, lo):
    """eq. (3.5): theta < 1 independent of h.  Energy-norm error reduction of
    V(2,2) red-black Gauss-Seidel on A e = 0 after a few cycles."""
    hier = O.build_hierarchy(dim, H, r)
    thetas = []
    for k in range(lo, r + 2):
        lev = hier.level(k)
        u = np.random.default_rng(0).standard_normal(lev.A.shape[0])
        z = np.zeros_like(u)
        prev = None
        for _ in range(8):
            u = O.vcycle(hier, k, z, u)
            e = O.energy_norm(lev, u)
            if prev is not None:
                ratio = e / prev
            prev = e
        thetas.append(ratio)
    assert max(thetas) < 0.3
    assert max(thetas[-2:]) / min(thetas[-2:]) < 1.1


# ---------------------------------------------------------------------------
# Closed-form discrete solution: f(u) = c u, u* = prod sin(pi x_i)
# ---------------------------------------------------------------------------


def closed_form_lambda(dim, h, c):
    """A_h s = mu s for the nodal sine s; the lumped discrete problem then has
    U = lambda s with lambda = h^d (d pi^2 + c) / (mu + c h^d)."""
    mu = (4 * dim * math.sin(math.pi * h / 2) ** 2) * h ** (dim - 2)
    return h ** dim * (dim * math.pi ** 2 + c) / (mu + c * h ** dim)


@pytest.mark.parametrize("dim,H,r", [(2, 4, 3), (3, 4, 2)])
def test_linear_case_closed_form(dim, H, r):
    c = 2.0
    prob = W.Problem(dim=dim, coarse_cells=H, refinements=r, f="linear", a=c,
                     modes=[((1,) * dim, 1.0)])
    hier = O.build_hierarchy(dim, H, r)
    g = prob.g_nodal()
    lev = hier.level(r + 1)
    exact = closed_form_lambda(dim, lev.h, c) * O.from_nodal(lev, prob.u_star())
    G = O.load_vector(lev, g)
    Ub, _ = O.newton_full(lev, G, "linear", c)
    np.testing.assert_allclose(Ub, exact, rtol=0, atol=1e-13)
    # many correction steps drive the FMG iterate onto the discrete solution
    res = O.fmg(hier, g, "linear", c, m=2, p=10)
    np.testing.assert_allclose(res.u[-1], exact, rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------
# Nonlinear solves
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("kind", ["cubic", "expm1", "signed_pow32", "neg_exp_neg"])
def test_full_newton_matches_root_finder(kind):
    lev = O.assemble_level(2, 8)
    rng = np.random.default_rng(5)
    G = lev.w * (3.0 + rng.standard_normal(lev.A.shape[0]))
    U, _ = O.newton_full(lev, G, kind, 1.0)
    Ad = lev.A.toarray()

    def F(x):
        return Ad @ x + lev.w * O.f_val(kind, 1.0, x) - G

    sol = opt.root(F, np.zeros_like(G), method="hybr", tol=1e-13)
    assert np.max(np.abs(F(sol.x))) < 1e-14
    np.testing.assert_allclose(U, sol.x, rtol=0, atol=1e-11)
    assert np.max(np.abs(F(U))) < 1e-15


def _step_setup(dim=2, H=4, r=2, kind="cubic"):
    prob = W.Problem(dim=dim, coarse_cells=H, refinements=r, f=kind, a=1.0,
                     modes=[((1, 2, 1)[:dim], 1.0), ((2, 1, 1)[:dim], -0.5)])
    hier = O.build_hierarchy(dim, H, r)
    k = r + 1
    lev = hier.level(k)
    G = O.load_vector(lev, prob.g_nodal())
    return prob, hier, k, lev, G


def test_augmented_solution_minimises_energy():
    """(3.6) is the Euler-Lagrange equation of the convex energy
    E(v) = a(v,v)/2 + sum_i w_i Phi(v_i) - (g, v) restricted to V_H + span{u~}."""
    prob, hier, k, lev, G = _step_setup()
    rng = np.random.default_rng(2)
    ut = O.newton_full(lev, G, prob.f, prob.a)[0] + 0.05 * rng.standard_normal(lev.A.shape[0])
    y, B, _ = O.augmented_newton(lev, hier.P_H[k - 1], ut, G, prob.f, prob.a)
    Ad = lev.A.toarray()
    Bd = B.toarray()

    def E(z):
        v = Bd @ z
        return 0.5 * v @ (Ad @ v) + lev.w @ O.f_antider(prob.f, prob.a, v) - G @ v

    z0 = np.zeros(B.shape[1])
    z0[-1] = 1.0
    sol = opt.minimize(E, z0, method="Powell", options={"xtol": 1e-12, "ftol": 1e-15, "maxiter": 200000})
    assert E(y) <= sol.fun + 1e-14
    np.testing.assert_allclose(Bd @ y, Bd @ sol.x, rtol=0, atol=1e-5)


def test_augmented_solution_is_basis_invariant():
    """V_H + span{u~} = V_H + span{u~ - P_{H->k} z}: the solution u is the same."""
    prob, hier, k, lev, G = _step_setup(kind="expm1")
    rng = np.random.default_rng(7)
    ut = O.newton_full(lev, G, prob.f, prob.a)[0] + 0.05 * rng.standard_normal(lev.A.shape[0])
    PH = hier.P_H[k - 1]
    y1, B1, _ = O.augmented_newton(lev, PH, ut, G, prob.f, prob.a)
    z = rng.standard_normal(PH.shape[1])
    y2, B2, _ = O.augmented_newton(lev, PH, ut - PH @ z, G, prob.f, prob.a)
    np.testing.assert_allclose(B1 @ y1, B2 @ y2, rtol=0, atol=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_correction_step_fixed_point(dim):
    """If u^(l) is the discrete solution, one correction step returns it."""
    prob, hier, k, lev, G = _step_setup(dim=dim, r=2 if dim == 2 else 1)
    ub, _ = O.newton_full(lev, G, prob.f, prob.a)
    u1, info = O.correction_step(hier, k, ub, G, prob.f, prob.a)
    np.testing.assert_allclose(u1, ub, rtol=0, atol=1e-12)
    assert abs(info.alpha - 1.0) < 1e-10 and np.max(np.abs(info.c)) < 1e-10


@pytest.mark.parametrize("kind", ["cubic", "expm1"])
def test_correction_step_contracts(kind):
    """Theorem 3.1: the energy error shrinks by gamma < 1 at every step."""
    prob, hier, k, lev, G = _step_setup(r=3, kind=kind)
    ub, _ = O.newton_full(lev, G, prob.f, prob.a)
    u = np.random.default_rng(4).standard_normal(lev.A.shape[0]) * 0.3
    errs = [O.energy_norm(lev, u - ub)]
    for _ in range(4):
        u, _ = O.correction_step(hier, k, u, G, prob.f, prob.a)
        errs.append(O.energy_norm(lev, u - ub))
    ratios = [errs[i + 1] / errs[i] for i in range(4)]
    assert max(ratios) < 0.3


# ---------------------------------------------------------------------------
# Full multigrid (Algorithm 3.2; Theorem 3.2; Corollary 3.1)
# ---------------------------------------------------------------------------


def test_fmg_optimal_orders_small_2d():
    """Corollary 3.1: L2 error O(h^2) and energy error O(h) at every level."""
    prob = W.config_small_2d()
    hier = O.build_hierarchy(2, prob.coarse_cells, prob.refinements)
    res = O.fmg(hier, prob.g_nodal(), prob.f, prob.a)
    l2, h1 = [], []
    for k in range(1, prob.levels + 1):
        a, b = O.fe_errors(hier.level(k), res.u[k - 1], prob)
        l2.append(a)
        h1.append(b)
    rl2 = [math.log2(l2[i] / l2[i + 1]) for i in range(len(l2) - 1)]
    rh1 = [math.log2(h1[i] / h1[i + 1]) for i in range(len(h1) - 1)]
    assert all(abs(r - 2.0) < 0.1 for r in rl2[1:]), rl2
    assert all(abs(r - 1.0) < 0.1 for r in rh1[1:]), rh1


def _two_mode_problem(dim, H, r, kind):
    return W.Problem(dim=dim, coarse_cells=H, refinements=r, f=kind, a=1.0,
                     modes=[((1,) * dim, 1.0), ((2, 1, 3)[:dim], 0.5)])


@pytest.mark.parametrize("make,m", [
    (lambda: _two_mode_problem(2, 4, 4, "cubic"), 2),
    (lambda: _two_mode_problem(2, 8, 3, "cubic"), 2),
    (lambda: _two_mode_problem(3, 4, 2, "expm1"), 2),
    (lambda: _two_mode_problem(3, 4, 3, "expm1"), 3),
    (lambda: W.config_3d(seed=0, refinements=3), 3),
])
def test_fmg_reaches_discretization_accuracy(make, m):
    """Theorem 3.2: ||u_bar_h - u_h|| stays a fraction of the discretization
    error; read as algebraic error <= 0.1 x discretization error (discrete L2)
    at every level.  On the cube the bar needs m = 3 cycles per step from 3
    refinements on (the 3D workloads' setting)."""
    prob = make()
    dim, r = prob.dim, prob.refinements
    hier = O.build_hierarchy(dim, prob.coarse_cells, r)
    g = prob.g_nodal()
    res = O.fmg(hier, g, prob.f, prob.a, m=m)
    for k in range(2, r + 2):
        lev = hier.level(k)
        G = O.load_vector(lev, O.restrict_nodal(g, dim, prob.n_fine, lev.n))
        ub, _ = O.newton_full(lev, G, prob.f, prob.a, U0=res.u[k - 1])
        e_alg = O.discrete_l2(lev, res.u[k - 1] - ub)
        e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star(lev.n)))
        assert e_alg <= 0.1 * e_disc, (k, e_alg, e_disc)


@pytest.mark.parametrize("dim,hf,Hs", [(2, 64, (2, 4, 8)), (3, 16, (2, 4))])
def test_correction_contraction_satisfies_theorem_3_2(dim, hf, Hs):
    """Theorem 3.1 / 3.2: the energy-error contraction gamma of one correction step (m = 2
    V(2,2) cycles, then the augmented problem), measured from random starts at a fixed fine
    mesh for several H, satisfies gamma^p beta < 1 with p = 1, beta = 2 -- with a wide margin:
    gamma is about theta^2 (two cycles at theta ~ 0.19), and it does not grow as H shrinks."""
    gammas = []
    for H in Hs:
        r = int(round(math.log2(hf / H)))
        prob = _two_mode_problem(dim, H, r, "cubic")
        hier = O.build_hierarchy(dim, H, r)
        lev = hier.level(r + 1)
        G = O.load_vector(lev, prob.g_nodal())
        ub, _ = O.newton_full(lev, G, prob.f, prob.a)
        worst = 0.0
        for seed in range(2):
            u = ub + 0.3 * np.random.default_rng(seed).standard_normal(ub.shape)
            e0 = O.energy_norm(lev, u - ub)
            for _ in range(2):
                u, _ = O.correction_step(hier, r + 1, u, G, prob.f, prob.a)
                e1 = O.energy_norm(lev, u - ub)
                worst = max(worst, e1 / e0)
                e0 = e1
        gammas.append(worst)
    assert all(2.0 * g < 1.0 for g in gammas)
    assert max(gammas) < 0.1
    assert gammas[-1] <= gammas[0] + 1e-3


def test_3d_with_two_cycles_misses_the_accuracy_bar():
    """The reason the 3D workloads take m = 3: with the paper's m = 2 the algebraic error on
    the cube passes a tenth of the discretization error at 3 refinements."""
    prob = W.config_3d(seed=0, refinements=3)
    hier = O.build_hierarchy(3, 4, 3)
    g = prob.g_nodal()
    res = O.fmg(hier, g, prob.f, prob.a, m=2)
    lev = hier.level(4)
    G = O.load_vector(lev, g)
    ub, _ = O.newton_full(lev, G, prob.f, prob.a, U0=res.u[-1])
    e_alg = O.discrete_l2(lev, res.u[-1] - ub)
    e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star()))
    assert e_alg > 0.1 * e_disc
    assert W.M_VCYCLES_3D == 3 and prob.m_vcycles == 3


@pytest.mark.parametrize("make,m", [
    (W.config_small_2d, 2),
    (lambda: W.config_large_2d(seed=0, refinements=4), 2),
    (lambda: _two_mode_problem(3, 4, 3, "expm1"), 2),
    (lambda: W.config_3d(seed=0, refinements=3), 3),
])
def test_newton_stopping_rule_gives_the_tight_tolerance_result(make, m):
    """The reading of the stopping rule the paper leaves open (Newton on eq. 3.6 and on level 1
    stops after the update whose increment is <= 1e-6 max(1, ||y||)): Newton's quadratic
    convergence leaves an error of order 1e-12 after that update, so the full multigrid
    result is the one a 1e-13 tolerance gives, to 1e-11 relative in the max norm."""
    prob = make()
    hier = O.build_hierarchy(prob.dim, prob.coarse_cells, prob.refinements)
    g = prob.g_nodal()
    loose = O.fmg(hier, g, prob.f, prob.a, m=m)
    tight = O.fmg(hier, g, prob.f, prob.a, m=m, tol=1e-13, tol_level1=1e-13)
    a, b = loose.u[-1], tight.u[-1]
    assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(b))
    # the tight rule takes at least as many iterations on every level
    assert all(sb.newton_iters >= sa.newton_iters for (_, sa), (_, sb) in zip(loose.steps, tight.steps))


def test_level_one_is_exact():
    """Algorithm 3.2 step 1 solves the semilinear problem on V_{h_1} exactly."""
    prob = W.config_small_2d()
    hier = O.build_hierarchy(2, 4, 1)
    g = prob.g_nodal(8)
    res = O.fmg(hier, g, prob.f, prob.a)
    lev = hier.level(1)
    G = O.load_vector(lev, O.restrict_nodal(g, 2, 8, 4))
    assert np.max(np.abs(O.nonlinear_residual(lev, G, prob.f, prob.a, res.u[0]))) < 1e-14


# ---------------------------------------------------------------------------
# Chebyshev-Jacobi smoother (the colour-free alternative smoother)
# ---------------------------------------------------------------------------


def _mode_vector(lev, kv):
    """Nodal sine mode prod_ax sin(k_ax pi x_ax) on the unknowns of a level: an eigenvector
    of the 2d+1-point stiffness with D^{-1}A eigenvalue 1 - mean_ax cos(k_ax pi h)."""
    X = lev.nodes[lev.interior] * lev.h
    v = np.ones(X.shape[0])
    for ax in range(lev.dim):
        v *= np.sin(kv[ax] * math.pi * X[:, ax])
    lam = 1.0 - np.mean([math.cos(k * math.pi * lev.h) for k in kv])
    return v, lam


@pytest.mark.parametrize("dim,n,kv", [(2, 16, (1, 1)), (2, 16, (7, 12)), (2, 16, (15, 15)), (3, 8, (2, 5, 7))])
@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_chebyshev_error_polynomial(dim, n, kv, degree):
    """After `degree` steps on A u = 0 the error is p(lam) e0 with the shifted, scaled
    Chebyshev polynomial p(lam) = T_k((theta - lam)/delta) / T_k(theta/delta) (evaluated
    here with numpy's Chebyshev series, not the smoother's recurrence)."""
    lev = O.assemble_level(dim, n)
    e0, lam = _mode_vector(lev, kv)
    u = e0.copy()
    O.chebyshev_smooth(lev, np.zeros_like(u), u, degree)
    lmin = O.CHEB_LMAX / O.CHEB_RATIO
    theta, delta = 0.5 * (O.CHEB_LMAX + lmin), 0.5 * (O.CHEB_LMAX - lmin)
    coef = np.zeros(degree + 1)
    coef[degree] = 1.0
    p = np.polynomial.chebyshev.chebval((theta - lam) / delta, coef) / np.polynomial.chebyshev.chebval(
        theta / delta, coef)
    assert np.allclose(u, p * e0, rtol=0, atol=1e-12 * np.max(np.abs(e0)))


def test_chebyshev_degree_one_is_damped_jacobi():
    lev = O.assemble_level(2, 8)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(lev.A.shape[0])
    u0 = rng.standard_normal(lev.A.shape[0])
    u = u0.copy()
    O.chebyshev_smooth(lev, b, u, 1)
    omega = 1.0 / (0.5 * (O.CHEB_LMAX + O.CHEB_LMAX / O.CHEB_RATIO))
    assert np.allclose(u, u0 + omega * (b - lev.A @ u0) / lev.diag, rtol=1e-14, atol=1e-14)


def test_chebyshev_damps_the_upper_spectrum():
    """The smoothing factor: every mode with D^{-1}A eigenvalue in [lmax/ratio, 2) is
    reduced at least by 1 / T_k(theta/delta) for degree k."""
    lev = O.assemble_level(2, 16)
    degree = 2
    lmin = O.CHEB_LMAX / O.CHEB_RATIO
    theta, delta = 0.5 * (O.CHEB_LMAX + lmin), 0.5 * (O.CHEB_LMAX - lmin)
    bound = 1.0 / math.cosh(degree * math.acosh(theta / delta))
    worst = 0.0
    for kx in range(1, 16):
        for ky in range(1, 16):
            e0, lam = _mode_vector(lev, (kx, ky))
            if lam < lmin:
                continue
            u = e0.copy()
            O.chebyshev_smooth(lev, np.zeros_like(u), u, degree)
            worst = max(worst, np.linalg.norm(u) / np.linalg.norm(e0))
    assert worst <= bound * (1 + 1e-12)


@pytest.mark.parametrize("dim,H,r,lo", [(2, 4, 5, 4), (3, 4, 4, 4)])
def test_chebyshev_vcycle_contraction_is_mesh_independent(dim, H, r, lo):
    hier = O.build_hierarchy(dim, H, r)
    thetas = []
    for k in range(lo, r + 2):
        lev = hier.level(k)
        u = np.random.default_rng(0).standard_normal(lev.A.shape[0])
        z = np.zeros_like(u)
        prev = None
        for _ in range(8):
            u = O.vcycle(hier, k, z, u, smoother="chebyshev")
            e = O.energy_norm(lev, u)
            if prev is not None:
                ratio = e / prev
            prev = e
        thetas.append(ratio)
    assert max(thetas) < 0.5
    assert max(thetas[-2:]) / min(thetas[-2:]) < 1.1


@pytest.mark.parametrize("dim,H,r,kind,m", [(2, 4, 4, "cubic", 2), (3, 4, 2, "expm1", 3)])
def test_fmg_with_chebyshev_reaches_discretization_accuracy(dim, H, r, kind, m):
    """With degree-2 Chebyshev smoothing the 3D V-cycle contracts by about 0.33 (red-black
    Gauss-Seidel: 0.26), so the 3D case takes m = 3 cycles per correction step."""
    prob = W.Problem(dim=dim, coarse_cells=H, refinements=r, f=kind, a=1.0,
                     modes=[((1,) * dim, 1.0), ((2, 1, 3)[:dim], 0.5)])
    hier = O.build_hierarchy(dim, H, r)
    g = prob.g_nodal()
    res = O.fmg(hier, g, prob.f, prob.a, m=m, smoother="chebyshev")
    lev = hier.level(r + 1)
    ub, _ = O.newton_full(lev, O.load_vector(lev, g), prob.f, prob.a, U0=res.u[-1])
    e_alg = O.discrete_l2(lev, res.u[-1] - ub)
    e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star()))
    assert e_alg <= 0.1 * e_disc, (e_alg, e_disc)


# ---------------------------------------------------------------------------
# Fixed-point variant of the augmented solve (the other nonlinear solver the paper names)
# ---------------------------------------------------------------------------


def test_augmented_fixed_point_reaches_the_newton_solution():
    prob, hier, k, lev, G = _step_setup()
    rng = np.random.default_rng(3)
    ut = O.newton_full(lev, G, prob.f, prob.a)[0] + 0.05 * rng.standard_normal(lev.A.shape[0])
    yn, B, _ = O.augmented_newton(lev, hier.P_H[k - 1], ut, G, prob.f, prob.a, tol=1e-13)
    yf, _, it = O.augmented_fixed_point(lev, hier.P_H[k - 1], ut, G, prob.f, prob.a, tol=1e-13)
    assert it > 3   # linear convergence: more iterations than Newton's
    assert np.max(np.abs(B @ yf - B @ yn)) <= 1e-11 * np.max(np.abs(B @ yn))


def test_augmented_fixed_point_contracts_at_the_linear_rate():
    """f(u) = c u: the fixed-point map is affine, y_{k+1} - y* = -K^{-1} (c B^T W B)(y_k - y*), so
    the increments shrink by the spectral radius of that matrix (from scipy's eigensolver)."""
    c = 10.0
    prob = W.Problem(dim=2, coarse_cells=4, refinements=2, f="linear", a=c, modes=[((1, 1), 1.0)])
    hier = O.build_hierarchy(2, 4, 2)
    k = 3
    lev = hier.level(k)
    G = O.load_vector(lev, prob.g_nodal())
    rng = np.random.default_rng(8)
    ut = rng.standard_normal(lev.A.shape[0])
    B = sp.hstack([hier.P_H[k - 1], sp.csr_matrix(ut[:, None])]).tocsr()
    K = (B.T @ (lev.A @ B)).toarray()
    Mw = (B.T @ (sp.diags(lev.w * c) @ B)).toarray()
    rho = max(abs(np.linalg.eigvals(np.linalg.solve(K, Mw))))
    assert 0.05 < rho < 0.9
    deltas = []
    y = np.zeros(B.shape[1])
    y[-1] = 1.0
    Gaug = B.T @ G
    for _ in range(12):
        y_new = np.linalg.solve(K, Gaug - B.T @ (lev.w * O.f_val("linear", c, B @ y)))
        deltas.append(np.linalg.norm(y_new - y))
        y = y_new
    assert abs(deltas[-1] / deltas[-2] - rho) < 1e-3 * rho
    # and the oracle's iteration takes the same steps
    yf, _, it = O.augmented_fixed_point(lev, hier.P_H[k - 1], ut, G, "linear", c, tol=1e-13, maxit=1000)
    exact = B @ np.linalg.solve(K + Mw, Gaug)
    assert np.max(np.abs(B @ yf - exact)) <= 1e-10 * np.max(np.abs(exact))


def test_fmg_with_fixed_point_reaches_discretization_accuracy():
    prob = W.Problem(dim=2, coarse_cells=4, refinements=4, f="cubic", a=1.0,
                     modes=[((1, 1), 1.0), ((2, 1), 0.5)])
    hier = O.build_hierarchy(2, 4, 4)
    g = prob.g_nodal()
    res = O.fmg(hier, g, prob.f, prob.a, nonlinear="fixed_point")
    newton = O.fmg(hier, g, prob.f, prob.a)
    lev = hier.level(5)
    ub, _ = O.newton_full(lev, O.load_vector(lev, g), prob.f, prob.a, U0=res.u[-1])
    e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star()))
    assert O.discrete_l2(lev, res.u[-1] - ub) <= 0.1 * e_disc
    assert O.discrete_l2(lev, res.u[-1] - newton.u[-1]) <= 1e-3 * e_disc
    assert sum(i.newton_iters for _, i in res.steps) > sum(i.newton_iters for _, i in newton.steps)


# ---------------------------------------------------------------------------
# The chord iteration (the mixed path's reading of the nonlinear solver of eq. (3.6), which the
# paper leaves open after Theorem 3.2): Newton's fixed point, reached at a linear rate
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("make", [lambda: W.config_large_2d(seed=0, refinements=5),
                                  lambda: W.config_3d(seed=0, refinements=3)])
def test_chord_fmg_matches_newton_fmg(make):
    """Algorithm 3.2 with the chord iteration gives Newton's result to rounding, and takes at
    most one more iteration per correction step."""
    prob = make()
    hier = O.build_hierarchy(prob.dim, prob.coarse_cells, prob.refinements)
    g = prob.g_nodal()
    rn = O.fmg(hier, g, prob.f, prob.a)
    rc = O.fmg(hier, g, prob.f, prob.a, nonlinear="chord")
    rel = np.max(np.abs(rn.u[-1] - rc.u[-1])) / np.max(np.abs(rn.u[-1]))
    assert rel <= 1e-11
    for (kn, sn), (kc, sc) in zip(rn.steps, rc.steps):
        assert kn == kc and sn.newton_iters <= sc.newton_iters <= sn.newton_iters + 1


def test_chord_is_slower_than_newton_far_from_the_solution():
    """From a far start on a strong nonlinearity the chord step (Jacobian of the first iterate)
    needs more iterations than Newton, and reaches the same (c, alpha)."""
    prob = W.config_large_2d(seed=0, refinements=3)
    hier = O.build_hierarchy(2, 8, 3)
    k = 4
    lev = hier.level(k)
    G = O.load_vector(lev, prob.g_nodal())
    a = 30.0
    ub, _ = O.newton_full(lev, G, "cubic", a)
    u0 = ub + 0.3 * np.random.default_rng(0).standard_normal(ub.shape)
    un, n_info = O.correction_step(hier, k, u0, G, "cubic", a, nonlinear="newton")
    uc, c_info = O.correction_step(hier, k, u0, G, "cubic", a, nonlinear="chord")
    assert c_info.newton_iters > n_info.newton_iters
    assert abs(c_info.alpha - n_info.alpha) <= 1e-7
    assert np.max(np.abs(uc - un)) <= 1e-7 * np.max(np.abs(un))


# ---------------------------------------------------------------------------
# Variable SPD coefficient A(x) of eq. (2.1): diagonal, constant on each cell of T_H
# ---------------------------------------------------------------------------


def _cell_coefficient(dim, nc, seed=3):
    return W.cell_coefficient(dim, nc, seed)


@pytest.mark.parametrize("dim,nc,r", [(2, 4, 3), (3, 2, 2)])
def test_coefficient_keeps_the_galerkin_identity(dim, nc, r):
    """With A constant on each cell of T_H every level discretizes the same bilinear form on
    nested P1 spaces, so A_{k-1} = P_k^T A_k P_k holds exactly (as for A = I)."""
    hier = O.build_hierarchy(dim, nc, r, coef=_cell_coefficient(dim, nc))
    for k in range(2, r + 2):
        A, P, Ac = hier.level(k).A, hier.level(k).P, hier.level(k - 1).A
        assert abs(P.T @ A @ P - Ac).max() <= 1e-13 * abs(Ac).max()


@pytest.mark.parametrize("dim,nc,n", [(2, 4, 16), (3, 2, 8)])
def test_coefficient_energy_of_linear_functions(dim, nc, n):
    """a(u, u) = sum_K |K| grad(u).A_K grad(u): for u = g.x (boundary nodes included) that is
    sum over the cells of T_H of |cell| sum_a A_a g_a^2, in closed form."""
    coef = _cell_coefficient(dim, nc)
    lev = O.assemble_level(dim, n, coef=coef, coef_cells=nc)
    g = np.random.default_rng(7).standard_normal(dim)
    u = (lev.nodes.astype(np.float64) / n) @ g
    exact = np.sum(coef * g ** 2) / nc ** dim
    assert abs(u @ (lev.S @ u) - exact) <= 1e-13 * exact


@pytest.mark.parametrize("dim,nc,n", [(2, 4, 16), (3, 2, 8)])
def test_coefficient_stiffness_is_an_axis_stencil(dim, nc, n):
    """A diagonal A keeps the couplings of the right-triangle and Kuhn meshes on the axis
    edges: only 2d+1 entries per row, non-positive off the diagonal, zero row sums over all
    nodes; A = c I scales the textbook stencil by c."""
    coef = _cell_coefficient(dim, nc)
    lev = O.assemble_level(dim, n, coef=coef, coef_cells=nc)
    S = lev.S.tocoo()
    dist = np.abs(lev.nodes[S.row] - lev.nodes[S.col]).sum(axis=1)
    assert np.all(dist <= 1)
    assert np.all(S.data[dist == 1] < 0)
    assert np.max(np.abs(np.asarray(lev.S.sum(axis=1)))) <= 1e-13 * np.abs(lev.S.diagonal()).max()
    c = np.full((nc ** dim, dim), 1.7)
    A1 = O.assemble_level(dim, n).A
    Ac = O.assemble_level(dim, n, coef=c, coef_cells=nc).A
    assert abs(Ac - 1.7 * A1).max() <= 1e-13 * abs(Ac).max()


@pytest.mark.parametrize("dim,nc,r", [(2, 8, 3), (3, 4, 2)])
def test_fmg_with_coefficient_reaches_discretization_accuracy(dim, nc, r):
    """Theorem 3.2 with a variable coefficient: the algebraic error stays below a tenth of the
    discretization error, estimated by Richardson as ||u_bar_h - P u_bar_2h|| / 3 (random-mode g,
    no closed-form solution)."""
    coef = _cell_coefficient(dim, nc)
    prob = W.Problem(dim=dim, coarse_cells=nc, refinements=r, f="cubic", a=1.0,
                     g_modes=[((1,) * dim, 3.0), ((2, 1, 3)[:dim], -2.0)])
    hier = O.build_hierarchy(dim, nc, r, coef=coef)
    g = prob.g_nodal()
    res = O.fmg(hier, g, prob.f, prob.a)
    lev, levc = hier.level(r + 1), hier.level(r)
    ub, _ = O.newton_full(lev, O.load_vector(lev, g), prob.f, prob.a, U0=res.u[-1])
    ubc, _ = O.newton_full(levc, O.load_vector(levc, O.restrict_nodal(g, dim, prob.n_fine, levc.n)), prob.f, prob.a)
    e_disc = O.discrete_l2(lev, ub - lev.P @ ubc) / 3.0
    assert O.discrete_l2(lev, res.u[-1] - ub) <= 0.1 * e_disc

"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case patches one step of the oracle with a plausible error and checks
that the corresponding pin quantity moves far outside its tolerance.
"""
import math

import numpy as np
import pytest

from oracle import fmg_oracle as O
from paper_1611_05677_gb300 import workloads as W


def _closed_form_error(dim=2, H=4, r=2, c=2.0):
    prob = W.Problem(dim=dim, coarse_cells=H, refinements=r, f="linear", a=c, modes=[((1,) * dim, 1.0)])
    hier = O.build_hierarchy(dim, H, r)
    lev = hier.level(r + 1)
    h = lev.h
    mu = 4 * dim * math.sin(math.pi * h / 2) ** 2 * h ** (dim - 2)
    lam = h ** dim * (dim * math.pi ** 2 + c) / (mu + c * h ** dim)
    res = O.fmg(hier, prob.g_nodal(), "linear", c, m=2, p=10)
    return float(np.max(np.abs(res.u[-1] - lam * O.from_nodal(lev, prob.u_star()))))


def test_unmutated_baseline():
    assert _closed_form_error() < 1e-12


def test_dropped_quadrature_weight_is_caught(monkeypatch):
    monkeypatch.setattr(O, "load_vector", lambda lev, g: g.ravel()[lev.interior])
    assert _closed_form_error() > 1e-3


def test_wrong_coarse_correction_sign_is_caught(monkeypatch):
    orig = O.prolongation

    def bad(dim, nc):
        P = orig(dim, nc).tolil()
        P[0, :] = -P[0, :]          # one wrong row
        return P.tocsr()

    monkeypatch.setattr(O, "prolongation", bad)
    Ac = O.assemble_level(2, 4).A
    Af = O.assemble_level(2, 8).A
    P = O.prolongation(2, 4)
    assert abs(P.T @ Af @ P - Ac).max() > 0.1


def test_dropped_nonlinear_term_in_linearized_rhs_is_caught(monkeypatch):
    """Algorithm 3.1 step 1 without -(f(x,u),v): the augmented solve still fixes
    the answer only up to the V_H + span{u~} approximation, so the FMG result
    drifts from the discrete solution beyond the accuracy criterion."""
    # patch the correction step to skip the nonlinear RHS term
    def bad_step(hier, k, u, G, kind, a, m=2, nu_pre=2, nu_post=2, tol=1e-12, smoother="rbgs", nonlinear="newton"):
        lev = hier.level(k)
        b = G.copy()
        ut = u.copy()
        for _ in range(m):
            ut = O.vcycle(hier, k, b, ut, nu_pre, nu_post)
        y, B, it = O.augmented_newton(lev, hier.P_H[k - 1], ut, G, kind, a, tol)
        return B @ y, O.StepInfo(newton_iters=it)

    prob = W.Problem(dim=2, coarse_cells=4, refinements=3, f="cubic", a=1.0,
                     modes=[((1, 1), 1.0), ((2, 1), 0.5)])
    hier = O.build_hierarchy(2, 4, 3)
    g = prob.g_nodal()
    lev = hier.level(4)
    G = O.load_vector(lev, g)
    ub, _ = O.newton_full(lev, G, prob.f, prob.a)
    good = O.fmg(hier, g, prob.f, prob.a).u[-1]
    monkeypatch.setattr(O, "correction_step", bad_step)
    bad = O.fmg(hier, g, prob.f, prob.a).u[-1]
    e_disc = O.discrete_l2(lev, ub - O.from_nodal(lev, prob.u_star()))
    assert O.discrete_l2(lev, good - ub) <= 0.1 * e_disc
    assert O.discrete_l2(lev, bad - ub) > 1.0 * e_disc


def test_wrong_chebyshev_coefficient_is_caught(monkeypatch):
    """A Chebyshev step that reuses the previous rho in the momentum term (a plausible slip
    in the three-term recurrence) no longer gives the Chebyshev error polynomial."""
    def bad(lev, b, u, degree, lmax=O.CHEB_LMAX, ratio=O.CHEB_RATIO):
        lmin = lmax / ratio
        theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
        sig = theta / delta
        rho = 1.0 / sig
        d = (b - lev.A @ u) / lev.diag / theta
        u += d
        for _ in range(1, degree):
            r = (b - lev.A @ u) / lev.diag
            rho_new = 1.0 / (2.0 * sig - rho)
            d = rho * rho * d + (2.0 * rho_new / delta) * r     # planted: rho instead of rho_new
            rho = rho_new
            u += d

    lev = O.assemble_level(2, 16)
    X = lev.nodes[lev.interior] * lev.h
    e0 = np.sin(7 * math.pi * X[:, 0]) * np.sin(12 * math.pi * X[:, 1])
    lam = 1.0 - 0.5 * (math.cos(7 * math.pi * lev.h) + math.cos(12 * math.pi * lev.h))
    lmin = O.CHEB_LMAX / O.CHEB_RATIO
    theta, delta = 0.5 * (O.CHEB_LMAX + lmin), 0.5 * (O.CHEB_LMAX - lmin)
    coef = np.array([0.0, 0.0, 0.0, 1.0])
    p = np.polynomial.chebyshev.chebval((theta - lam) / delta, coef) / np.polynomial.chebyshev.chebval(
        theta / delta, coef)
    good = e0.copy()
    O.chebyshev_smooth(lev, np.zeros_like(e0), good, 3)
    assert np.max(np.abs(good - p * e0)) < 1e-12
    monkeypatch.setattr(O, "chebyshev_smooth", bad)
    u = e0.copy()
    O.chebyshev_smooth(lev, np.zeros_like(e0), u, 3)
    assert np.max(np.abs(u - p * e0)) > 1e-3 * np.max(np.abs(e0))


def _far_start_iterations(a=30.0):
    prob = W.config_large_2d(seed=0, refinements=3)
    hier = O.build_hierarchy(2, 8, 3)
    k = 4
    lev = hier.level(k)
    G = O.load_vector(lev, prob.g_nodal())
    ub, _ = O.newton_full(lev, G, "cubic", a)
    u0 = ub + 0.3 * np.random.default_rng(0).standard_normal(ub.shape)
    _, n_info = O.correction_step(hier, k, u0, G, "cubic", a, nonlinear="newton")
    _, c_info = O.correction_step(hier, k, u0, G, "cubic", a, nonlinear="chord")
    return n_info.newton_iters, c_info.newton_iters


def test_chord_that_refactors_every_step_is_caught(monkeypatch):
    """A 'chord' step that assembles the Jacobian at every iterate is Newton: the far-start pin
    (chord strictly slower than Newton) no longer holds."""
    n, c = _far_start_iterations()
    assert c > n
    monkeypatch.setattr(O, "augmented_chord", O.augmented_newton)
    n, c = _far_start_iterations()
    assert c == n


def test_chord_with_a_dropped_load_term_is_caught(monkeypatch):
    """A chord step whose residual omits B^T G converges to another fixed point: the FMG result
    moves far from Newton's."""
    orig = O.augmented_chord

    def bad(lev, PHk, ut, G, kind, a, tol=1e-6, maxit=30):
        return orig(lev, PHk, ut, 0.0 * G, kind, a, tol, maxit)

    prob = W.config_large_2d(seed=0, refinements=3)
    hier = O.build_hierarchy(2, 8, 3)
    g = prob.g_nodal()
    good = O.fmg(hier, g, prob.f, prob.a).u[-1]
    # unmutated: the chord result is Newton's up to the stopping rule's error (~1e-10 at this size)
    assert np.max(np.abs(O.fmg(hier, g, prob.f, prob.a, nonlinear="chord").u[-1] - good)) <= 1e-8 * np.max(np.abs(good))
    monkeypatch.setattr(O, "augmented_chord", bad)
    worse = O.fmg(hier, g, prob.f, prob.a, nonlinear="chord").u[-1]
    assert np.max(np.abs(worse - good)) > 1e-3 * np.max(np.abs(good))

"""The seeded input generators against their stated recipes.  The manufactured right-hand side
g = -Laplace(u*) + a f(u*) (closed form in the generator) is checked against a finite-difference
Laplacian of the generator's own u*, extrapolated to fourth order, with a f written out here from
the examples' definitions; the mode draws, the batched instances and the request stream against
their recipes (ranges, no repeated modes, distributions, reproducibility by seed)."""
import math

import numpy as np
import pytest

from paper_1611_05677_gb300 import workloads as W


def fd_laplacian(u, n):
    """Minus the (2d+1)-point finite-difference Laplacian at interior nodes, spacing 1/n."""
    d = u.ndim
    inner = (slice(1, -1),) * d
    lap = -2.0 * d * u[inner]
    for ax in range(d):
        lo = [slice(1, -1)] * d
        hi = [slice(1, -1)] * d
        lo[ax] = slice(0, -2)
        hi[ax] = slice(2, None)
        lap = lap + u[tuple(lo)] + u[tuple(hi)]
    return -lap * n * n


def minus_laplacian_extrapolated(prob, n):
    """-Laplace(u*) at the interior nodes of the n-grid, from the n- and 2n-grids (h^2 error
    terms cancel: (4 L_2n - L_n) / 3)."""
    coarse = fd_laplacian(prob.u_star(n), n)
    fine = fd_laplacian(prob.u_star(2 * n), 2 * n)
    every_other = (slice(1, None, 2),) * prob.dim
    return (4.0 * fine[every_other] - coarse) / 3.0


def a_f(kind, a, u):
    return {"cubic": a * u ** 3, "expm1": a * (np.exp(u) - 1.0)}[kind]


@pytest.mark.parametrize("make,n", [(W.config_small_2d, 64), (lambda: W.config_large_2d(seed=3), 128),
                                    (lambda: W.config_3d(seed=1), 64)])
def test_manufactured_g_is_minus_laplacian_plus_f(make, n):
    prob = make()
    u = prob.u_star(n)
    g = prob.g_nodal(n)
    inner = (slice(1, -1),) * prob.dim
    want = minus_laplacian_extrapolated(prob, n) + a_f(prob.f, prob.a, u[inner])
    scale = np.max(np.abs(g[inner]))
    assert np.max(np.abs(g[inner] - want)) <= 1e-5 * scale
    # x is the fastest axis: u* of a single mode sin(k pi x) sin(l pi y) varies along the last axis by k
    one = W.Problem(dim=2, coarse_cells=4, refinements=2, modes=[((1, 3), 1.0)])
    x = np.arange(17) / 16
    assert np.allclose(one.u_star()[8, :], np.sin(math.pi * x) * np.sin(3 * math.pi * 0.5))


def test_mode_draws_follow_the_recipe():
    for seed in range(5):
        p2 = W.config_large_2d(seed=seed)
        ks = [kv for kv, _ in p2.modes]
        assert len(ks) == 8 and len(set(ks)) == 8
        assert all(1 <= k <= 6 for kv in ks for k in kv)
        p3 = W.config_3d(seed=seed)
        assert all(len(kv) == 3 and all(1 <= k <= 4 for k in kv) for kv, _ in p3.modes)
        assert all(0.0 <= c <= 1.0 for _, c in p3.modes)
    assert W.config_large_2d(seed=7).modes == W.config_large_2d(seed=7).modes
    assert W.config_large_2d(seed=7).modes != W.config_large_2d(seed=8).modes


def test_batch_follows_the_recipe():
    batch = W.config_batch(seed=0)
    assert len(batch) == 256
    rs = [p.refinements for p in batch]
    assert set(rs) == set(range(5, 10))
    assert all(0.5 <= p.a <= 2.0 and p.coarse_cells == 4 and p.f == "cubic" for p in batch)
    assert all(p.modes is None and len(p.g_modes) == 8 for p in batch)
    # a random-mode g is the mode sum itself (no manufactured solution)
    p = batch[0]
    assert np.allclose(p.g_nodal(), p._mode_sum(p.g_modes, p.n_fine))


def test_request_stream_follows_the_recipe():
    reqs = W.request_stream(seed=0, count=2000, rate=200.0)
    t = np.array([a for a, _ in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0          # Poisson at 200 requests/s
    dims = np.array([p.dim for _, p in reqs])
    assert abs((dims == 2).mean() - 0.7) < 0.05
    assert all(5 <= p.refinements <= 10 for _, p in reqs if p.dim == 2)
    assert all(3 <= p.refinements <= 6 for _, p in reqs if p.dim == 3)
    assert {p.f for _, p in reqs} == {"cubic", "expm1"}

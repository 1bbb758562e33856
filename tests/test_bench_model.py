"""The bench's compulsory-traffic model of one FMG solve (bytes per fine DOF), against the
values it must give by hand: in 2D with m = 2 V(2,2) red-black cycles and three Newton passes,
a V-cycle costs (4 x 24 + 2 x 18) x 4/3 = 176 B per node of its top level in FP64, a
correction step 24 + 2 x 176 + 16 + 3 x 8 + 16 = 432 B and the FMG solve 432 x 4/3 = 576 B per
fine DOF; the mixed path's FP32 cycle costs 40 + (4 x 12 + 2 x 9) x 4/3 = 128 B, its step 336 B
and its solve 448 B per fine DOF."""
import pytest

import bench


def test_fp64_2d():
    assert bench.solve_bytes_per_dof(2, False, 2, "rbgs") == pytest.approx(576.0)


def test_mixed_2d():
    assert bench.solve_bytes_per_dof(2, True, 2, "rbgs") == pytest.approx(448.0)


def test_fp64_3d():
    # cycle (4 x 24 + 2 x 17) x 8/7, step 24 + 2 cycles + 56, solve x 8/7
    cycle = (96 + 34) * 8 / 7
    assert bench.solve_bytes_per_dof(3, False, 2, "rbgs") == pytest.approx((24 + 2 * cycle + 56) * 8 / 7)


def test_cycles_and_smoother_enter_linearly():
    one = bench.solve_bytes_per_dof(2, True, 1, "chebyshev")
    two = bench.solve_bytes_per_dof(2, True, 2, "chebyshev")
    three = bench.solve_bytes_per_dof(2, True, 3, "chebyshev")
    assert three - two == pytest.approx(two - one)
    # a Chebyshev step streams u, b, d and writes u, d: 20 B in FP32 against a sweep's 12
    assert two - bench.solve_bytes_per_dof(2, True, 2, "rbgs") == pytest.approx(2 * 4 * 8 * (4 / 3) ** 2)


def test_batch_richardson_prolongation_is_the_p1_interpolation():
    # the nodal P1 interpolation of the batch bench's Richardson estimate reproduces linear
    # functions, and at the midpoint of a cell's (0,0)-(1,1) diagonal it averages that
    # diagonal's ends (not the other two corners)
    import numpy as np

    import bench

    n = 8
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x)          # rows y, columns x: x fastest
    lin = 0.3 + 1.7 * X - 2.1 * Y
    xf = np.arange(2 * n + 1) / (2 * n)
    Xf, Yf = np.meshgrid(xf, xf)
    assert np.allclose(bench.prolong_2d(lin), 0.3 + 1.7 * Xf - 2.1 * Yf, atol=1e-14)
    e = np.zeros((n + 1, n + 1))
    e[2, 3] = 1.0                      # coarse node x = 3, y = 2
    f = bench.prolong_2d(e)
    assert f[5, 7] == 0.5 and f[3, 5] == 0.5   # diagonal midpoints towards (+1, +1) and (-1, -1)
    assert f[5, 5] == 0.0 and f[3, 7] == 0.0   # the other diagonal is not an edge


def test_serve_requests_get_their_own_g():
    # the serving bench writes each request's random-mode g from its separable factors; it is
    # the workload's own g (closed-form mode sum), 2D and 3D
    import numpy as np
    import torch

    import bench
    from paper_1611_05677_gb300 import workloads as W

    seen = set()
    for _, p in W.request_stream(seed=2, count=200):
        if p.n_fine > 128 or p.dim in seen:
            continue
        seen.add(p.dim)
        out = torch.empty((p.n_fine + 1,) * p.dim, dtype=torch.float64)
        bench.random_mode_g(p, out)
        assert np.max(np.abs(out.numpy() - p.g_nodal())) <= 1e-12
    assert seen == {2, 3}

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

"""Seeded synthetic inputs for the semilinear FMG solver.

This module only draws problem data: the manufactured solutions, the nodal
right-hand side g of  -Laplace(u) + a*f(u) = g  on the unit square / cube, and
the instance mixes of the batched and served workloads.  It holds none of the
multigrid or multilevel-correction arithmetic, so both the FP64 oracle and the
CUDA path can take their inputs from here without sharing any method code.

The problem class is the model problem of Sec. 2 (eq. 2.1) on Omega = (0,1)^d
with A = I, or with a diagonal SPD coefficient A(x) that is constant on each cell
of the coarsest mesh T_H (entries drawn here, see cell_coefficient); the nonlinearities are those of the examples of Sec. 4
(Example 1: u^3; Example 2: -exp(-u); Example 3: the odd extension of
u^{3/2}) plus exp(u)-1 and the linear a*u used as a closed-form test case.

Node layout of every nodal array: (n+1)^d entries including the boundary
ring, x fastest, node (i,j[,l]) at coordinates (i,j[,l])/n.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Nonlinearity names; the C-ABI enum uses the same order.
NONLINEARITIES = ("cubic", "expm1", "linear", "signed_pow32", "neg_exp_neg")


def _f_problem(kind: str, a: float, u: np.ndarray) -> np.ndarray:
    """a*f(u) for the manufactured right-hand side (problem data, not the method)."""
    if kind == "cubic":
        return a * u * u * u
    if kind == "expm1":
        return a * np.expm1(u)
    if kind == "linear":
        return a * u
    if kind == "signed_pow32":
        return a * np.sign(u) * np.abs(u) ** 1.5
    if kind == "neg_exp_neg":
        return -a * np.exp(-u)
    raise ValueError(f"unknown nonlinearity {kind!r}")


@dataclass
class Problem:
    """One semilinear instance on nested uniform meshes.

    dim            2 (right triangles) or 3 (Kuhn tetrahedra)
    coarse_cells   1/H, cells per side of the coarsest mesh T_H
    refinements    number of uniform refinements; levels 1..refinements+1
    f, a           nonlinearity name and scale (a > 0 keeps f monotone)
    modes          list of (wave-vector, amplitude) of the manufactured u*,
                   or None when g is given directly (random-mode g)
    g_modes        list of (wave-vector, amplitude) of a direct g (no u*)
    g_const        constant g (Example 2 uses g = 1)
    coefficient    None (A = I) or the (coarse_cells^dim, dim) table of A's diagonal
                   entries per cell of T_H (cell (cx, cy[, cz]) at row cx + nc cy [+ nc^2 cz])
    """

    dim: int
    coarse_cells: int
    refinements: int
    f: str = "cubic"
    a: float = 1.0
    modes: list | None = None
    g_modes: list | None = None
    g_const: float | None = None
    name: str = ""
    m_vcycles: int = 2
    nu_pre: int = 2
    nu_post: int = 2
    p_corrections: int = 1
    coefficient: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_fine(self) -> int:
        return self.coarse_cells << self.refinements

    @property
    def levels(self) -> int:
        return self.refinements + 1

    def cells(self, level: int) -> int:
        """Cells per side at level k (1-based; level 1 is the coarse mesh T_H)."""
        return self.coarse_cells << (level - 1)

    @property
    def fine_dofs(self) -> int:
        return (self.n_fine - 1) ** self.dim

    def coords(self, n: int | None = None) -> list[np.ndarray]:
        """Nodal coordinate arrays (each shaped (n+1,)*dim, x fastest in memory)."""
        n = self.n_fine if n is None else n
        x = np.arange(n + 1, dtype=np.float64) / n
        grids = np.meshgrid(*([x] * self.dim), indexing="ij")
        # meshgrid 'ij' gives axis 0 = x; transpose so that x is the LAST axis
        # of the C-ordered array (x fastest).
        return [g.transpose(tuple(range(self.dim))[::-1]) for g in grids]

    def _mode_sum(self, modes, n: int, weight=None) -> np.ndarray:
        """Sum over modes of c * prod_ax sin(k_ax pi x_ax) on the nodal grid (x fastest).

        Evaluated as outer products of 1D factors, multiplied in the order c, x, y[, z]."""
        x = np.arange(n + 1, dtype=np.float64) / n
        out = np.zeros((n + 1,) * self.dim)
        for kv, c in modes:
            amp = float(c) if weight is None else weight(kv, c)
            t = amp * np.sin(kv[0] * math.pi * x)
            for ax in range(1, self.dim):
                s_ax = np.sin(kv[ax] * math.pi * x)
                t = t[None, ...] * s_ax.reshape((-1,) + (1,) * t.ndim)
            out += t
        return out

    def u_star(self, n: int | None = None) -> np.ndarray | None:
        if self.modes is None:
            return None
        n = self.n_fine if n is None else n
        return self._mode_sum(self.modes, n)

    def grad_u_star(self, pts: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """u* and grad u* at points pts (M, dim); used for FE error norms."""
        val = np.zeros(pts.shape[0])
        grad = np.zeros_like(pts)
        for kv, c in self.modes:
            s = [np.sin(kv[ax] * math.pi * pts[:, ax]) for ax in range(self.dim)]
            co = [kv[ax] * math.pi * np.cos(kv[ax] * math.pi * pts[:, ax]) for ax in range(self.dim)]
            val += c * np.prod(s, axis=0)
            for ax in range(self.dim):
                t = np.full(pts.shape[0], float(c))
                for bx in range(self.dim):
                    t = t * (co[bx] if bx == ax else s[bx])
                grad[:, ax] += t
        return val, grad

    def g_nodal(self, n: int | None = None) -> np.ndarray:
        """Nodal g on the (n+1)^d grid (boundary entries included, not used)."""
        n = self.n_fine if n is None else n
        if self.modes is not None:
            # g = -Laplace(u*) + a f(u*) in closed form.
            lap = self._mode_sum(self.modes, n,
                                 weight=lambda kv, c: float(c) * math.pi ** 2 * float(sum(k * k for k in kv)))
            return np.ascontiguousarray(lap + _f_problem(self.f, self.a, self.u_star(n)))
        g = np.zeros((n + 1,) * self.dim)
        if self.g_modes is not None:
            g += self._mode_sum(self.g_modes, n)
        if self.g_const is not None:
            g += self.g_const
        return np.ascontiguousarray(g)


def cell_coefficient(dim: int, coarse_cells: int, seed: int = 3, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """A diagonal SPD coefficient constant on each cell of T_H: entries U[lo, hi] (contrast
    hi/lo = 4 between neighbouring cells and between the axes of one cell), shape
    (coarse_cells^dim, dim), x fastest over the cells."""
    return np.random.default_rng(seed).uniform(lo, hi, size=(coarse_cells ** dim, dim))


def _draw_modes(rng: np.random.Generator, dim: int, kmax: int, count: int, amp: str):
    grid = [tuple(int(v) for v in t) for t in np.ndindex(*([kmax] * dim))]
    pick = rng.choice(len(grid), size=count, replace=False)
    kvs = [tuple(k + 1 for k in grid[i]) for i in pick]
    if amp == "normal":
        cs = rng.standard_normal(count)
    else:
        cs = rng.uniform(0.0, 1.0, count)
    return [(kv, float(c)) for kv, c in zip(kvs, cs)]


def config_small_2d() -> Problem:
    """2D, H=1/4, 4 refinements (65x65 nodes), u^3, u* = sin(pi x) sin(pi y)."""
    return Problem(dim=2, coarse_cells=4, refinements=4, f="cubic", a=1.0,
                   modes=[((1, 1), 1.0)], name="2d_H4_r4_cubic_sin")


def config_large_2d(seed: int = 0, refinements: int = 8) -> Problem:
    """2D, H=1/8, 8 refinements (2049x2049 nodes), u^3, u* = 8 seeded sin modes, k,l in 1..6."""
    rng = np.random.default_rng(seed)
    return Problem(dim=2, coarse_cells=8, refinements=refinements, f="cubic", a=1.0,
                   modes=_draw_modes(rng, 2, 6, 8, "normal"),
                   name=f"2d_H8_r{refinements}_cubic_8modes_seed{seed}")


# Multigrid cycles per correction step on the cube.  With m = 2 the algebraic error of the 3D
# full multigrid solve grows past a tenth of the discretization error from 3 refinements on
# (0.10 at 3 refinements and rising per level), with m = 3 it stays near 0.03 (red-black
# Gauss-Seidel); Theorem 3.2 only bounds it, so m is raised for every 3D workload.
M_VCYCLES_3D = 3


def config_coefficient(dim: int = 2, seed: int = 0, refinements: int | None = None) -> Problem:
    """The 2D (H = 1/8) or 3D (H = 1/4) workload shape with the variable coefficient of
    cell_coefficient(seed = 3) and a random-mode g (no closed-form solution with a coefficient
    that jumps across the cells of T_H); 2D cubic, 3D exp(u) - 1."""
    rng = np.random.default_rng(seed)
    if dim == 2:
        r = 8 if refinements is None else refinements
        return Problem(dim=2, coarse_cells=8, refinements=r, f="cubic", a=1.0,
                       g_modes=_draw_modes(rng, 2, 6, 8, "normal"), coefficient=cell_coefficient(2, 8),
                       name=f"2d_H8_r{r}_cubic_coefficient_seed{seed}")
    r = 6 if refinements is None else refinements
    return Problem(dim=3, coarse_cells=4, refinements=r, f="expm1", a=1.0,
                   g_modes=_draw_modes(rng, 3, 4, 8, "uniform"), coefficient=cell_coefficient(3, 4),
                   m_vcycles=M_VCYCLES_3D, name=f"3d_H4_r{r}_expm1_coefficient_seed{seed}")


def config_3d(seed: int = 0, refinements: int = 6) -> Problem:
    """3D Kuhn, H=1/4, 6 refinements (257^3 nodes), exp(u)-1, 8 seeded modes, amplitudes U[0,1]."""
    rng = np.random.default_rng(seed)
    return Problem(dim=3, coarse_cells=4, refinements=refinements, f="expm1", a=1.0,
                   modes=_draw_modes(rng, 3, 4, 8, "uniform"), m_vcycles=M_VCYCLES_3D,
                   name=f"3d_H4_r{refinements}_expm1_8modes_seed{seed}")


def config_batch(seed: int = 0, count: int = 256, rmin: int = 5, rmax: int = 9) -> list[Problem]:
    """Independent 2D instances, H=1/4, refinements U{rmin..rmax}, a*u^3 with a~U[0.5,2], random-mode g."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        r = int(rng.integers(rmin, rmax + 1))
        a = float(rng.uniform(0.5, 2.0))
        gm = _draw_modes(rng, 2, 6, 8, "normal")
        out.append(Problem(dim=2, coarse_cells=4, refinements=r, f="cubic", a=a, g_modes=gm,
                           name=f"batch{i}_r{r}"))
    return out


def request_stream(seed: int = 0, count: int = 2200, rate: float = 200.0,
                   r2d=(5, 10), r3d=(3, 6), frac_2d: float = 0.7):
    """Poisson arrivals of mixed 2D/3D semilinear solves.

    Returns a list of (arrival_time_seconds, Problem).  70% 2D (refinements
    U{5..10} of H=1/4), 30% 3D (U{3..6} of H=1/4); f is u^3 or exp(u)-1 with
    equal probability; g is a seeded random-mode function.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        is2d = rng.uniform() < frac_2d
        dim = 2 if is2d else 3
        lo, hi = r2d if is2d else r3d
        r = int(rng.integers(lo, hi + 1))
        f = "cubic" if rng.uniform() < 0.5 else "expm1"
        gm = _draw_modes(rng, dim, 6 if is2d else 4, 8, "normal")
        out.append((t, Problem(dim=dim, coarse_cells=4, refinements=r, f=f, a=1.0, g_modes=gm,
                               m_vcycles=2 if is2d else M_VCYCLES_3D, name=f"req{i}_{dim}d_r{r}_{f}")))
    return out

"""FP64 CPU oracle of the full multigrid method for semilinear elliptic problems
(H. Xie and F. Xu, "A full multigrid method for semilinear elliptic equation",
arXiv 1611.05677).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  The CUDA solver never calls it and
shares no code, tables or helpers with it.

What it computes, step by step and in the paper's order, in FP64 with
assembled sparse matrices:

* Sec. 2, eq. (2.6)-(2.7): P1 finite elements on a simplicial mesh of
  (0,1)^d; element-by-element stiffness assembly from barycentric gradients;
  the L2 pairings (f(x,u),v) and (g,v) are taken with the vertex
  (mass-lumped) quadrature rule on the current mesh.
* Sec. 3, eq. (3.1)-(3.3): nested uniformly refined meshes (beta = 2,
  2D "/" right triangles, 3D Kuhn tetrahedra); the prolongation P_k is the
  matrix of the natural inclusion V_{h_{k-1}} -> V_{h_k}, built by evaluating
  the coarse basis at the fine nodes; restriction is P_k^T.
* Algorithm 3.1 step 1, eq. (3.4)-(3.5): the linearized boundary value problem
  with the nonlinearity frozen at the current iterate, solved by m V-cycles
  (red-black Gauss-Seidel smoothing, or Chebyshev-Jacobi smoothing as the colour-free
  alternative; exact solve on the coarsest mesh).
* Algorithm 3.1 step 2, eq. (3.6): the semilinear problem on
  V_{H,h_k} = V_H + span{u~}, solved by Newton's method on the assembled
  (N_H+1)-dimensional Galerkin system (the nonlinear iteration is left open
  by the paper after Theorem 3.2; Newton is one of the two it names).  The
  fixed-point iteration, the other one it names, and the chord (simplified
  Newton) iteration, the mixed-precision path's reading, are options.
* Algorithm 3.2: the full multigrid schedule (exact solve on V_{h_1}, then
  p correction steps per level).
* Brute force: Newton on the full discrete problem (2.7) with sparse direct
  solves, as the "exact" discrete solution u_bar_h.

Readings where the paper is silent (each is listed with its reason in the
design notes): h_1 = H; vertex quadrature; V(nu1,nu2) cycles with red->black
pre-smoothing and black->red post-smoothing; Newton on the augmented space
from (c, alpha) = (0, 1) stopping after the update whose increment satisfies
||delta||_inf <= tol*max(1,||y||_inf), tol = 1e-6 (quadratic convergence leaves
an error of order tol^2 = 1e-12 after that update); the same rule, from U = 0,
for the exact solve on level 1.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ---------------------------------------------------------------------------
# Nonlinearities f(x,u) (Sec. 4 examples); each is monotone for a > 0, which
# is the first condition of Assumption A (eq. 2.5).
# ---------------------------------------------------------------------------


def f_val(kind: str, a: float, u: np.ndarray) -> np.ndarray:
    if kind == "cubic":            # Example 1
        return a * u ** 3
    if kind == "expm1":            # exp(u) - 1
        return a * np.expm1(u)
    if kind == "linear":           # a*u: the linear special case with a closed form
        return a * u
    if kind == "signed_pow32":     # Example 3, odd extension of u^{3/2}
        return a * np.sign(u) * np.abs(u) ** 1.5
    if kind == "neg_exp_neg":      # Example 2: -exp(-u)
        return -a * np.exp(-u)
    raise ValueError(kind)


def f_der(kind: str, a: float, u: np.ndarray) -> np.ndarray:
    if kind == "cubic":
        return 3.0 * a * u ** 2
    if kind == "expm1":
        return a * np.exp(u)
    if kind == "linear":
        return np.full_like(u, a)
    if kind == "signed_pow32":
        return 1.5 * a * np.sqrt(np.abs(u))
    if kind == "neg_exp_neg":
        return a * np.exp(-u)
    raise ValueError(kind)


def f_antider(kind: str, a: float, u: np.ndarray) -> np.ndarray:
    """Phi with Phi' = f and Phi(0) = 0: the convex potential of the nonlinearity."""
    if kind == "cubic":
        return a * u ** 4 / 4.0
    if kind == "expm1":
        return a * (np.expm1(u) - u)
    if kind == "linear":
        return a * u ** 2 / 2.0
    if kind == "signed_pow32":
        return a * np.abs(u) ** 2.5 / 2.5
    if kind == "neg_exp_neg":
        return a * (np.exp(-u) - 1.0)
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# Meshes (Sec. 3, eq. 3.1): uniform Freudenthal/Kuhn triangulations.
# ---------------------------------------------------------------------------


def structured_mesh(dim: int, n: int):
    """Nodes (integer lattice coordinates, x fastest) and simplices of the
    uniform mesh with n cells per side.

    Every cell with lower corner v0 is split into dim! simplices, one per
    permutation pi of the axes, with vertices v0, v0+e_pi0, v0+e_pi0+e_pi1, ...
    In 2D this is the "/" split of each square along its (0,0)-(1,1) diagonal;
    in 3D it is the Kuhn subdivision into 6 tetrahedra.  Simplices are stored
    cell by cell, dim! consecutive entries per cell, permutations in
    itertools order.
    """
    ax = np.arange(n + 1)
    grids = np.meshgrid(*([ax] * dim), indexing="ij")
    # node id = i + (n+1) j (+ (n+1)^2 l): x fastest
    nodes = np.stack([g.transpose(tuple(range(dim))[::-1]).ravel() for g in grids], axis=1)
    stride = np.array([(n + 1) ** a for a in range(dim)])
    cax = np.arange(n)
    cgrids = np.meshgrid(*([cax] * dim), indexing="ij")
    corners = np.stack([g.transpose(tuple(range(dim))[::-1]).ravel() for g in cgrids], axis=1)
    perms = list(itertools.permutations(range(dim)))
    simp = np.empty((corners.shape[0], len(perms), dim + 1), dtype=np.int64)
    for pi_idx, pi in enumerate(perms):
        v = corners.copy()
        simp[:, pi_idx, 0] = v @ stride
        for s in range(dim):
            v = v.copy()
            v[:, pi[s]] += 1
            simp[:, pi_idx, s + 1] = v @ stride
    return nodes, simp.reshape(-1, dim + 1), perms


def interior_mask(nodes: np.ndarray, n: int) -> np.ndarray:
    return np.all((nodes > 0) & (nodes < n), axis=1)


def barycentric_gradients(X: np.ndarray):
    """For simplices with vertex coordinates X (M, d+1, d): gradients of the
    barycentric coordinates (M, d+1, d) and volumes (M,).

    With E = [v1-v0, ..., vd-v0] (columns), x = v0 + E lam', so
    grad lam_i = row i of E^{-1} (i >= 1) and grad lam_0 = -sum of the others.
    """
    E = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    Einv = np.linalg.inv(E)
    d = X.shape[2]
    grads = np.empty((X.shape[0], d + 1, d))
    grads[:, 1:, :] = Einv
    grads[:, 0, :] = -Einv.sum(axis=1)
    vol = np.abs(np.linalg.det(E)) / math.factorial(d)
    return grads, vol


@dataclass
class Level:
    """One level of the nested hierarchy: T_{h_k} with n cells per side."""

    dim: int
    n: int
    h: float
    nodes: np.ndarray          # (Nall, dim) lattice coordinates
    interior: np.ndarray       # (N,) node ids of the unknowns
    A: sp.csr_matrix           # stiffness on the unknowns, eq. (2.3)
    w: np.ndarray              # vertex-rule weights of the unknowns
    diag: np.ndarray = None
    Aoff: sp.csr_matrix = None
    red: np.ndarray = None     # positions (into the unknowns) of colour 0
    black: np.ndarray = None
    A_red: sp.csr_matrix = None
    A_black: sp.csr_matrix = None
    P: sp.csr_matrix = None    # prolongation from level k-1 (None on level 1)
    chol: tuple = None         # Cholesky factor of A on the coarsest level
    S: sp.csr_matrix = None    # stiffness on all nodes (boundary included)
    extra: dict = field(default_factory=dict)


def element_coefficients(coef: np.ndarray, dim: int, nc: int, Xs: np.ndarray) -> np.ndarray:
    """A on each element: the diagonal of the coarse cell of T_H (1/H = nc cells per side)
    that holds the element's centroid; coef has one row of d diagonal entries per coarse cell,
    x fastest."""
    cen = Xs.mean(axis=1)                                    # (M, d) centroids
    cell = np.minimum(np.floor(cen * nc).astype(np.int64), nc - 1)
    cid = cell @ np.array([nc ** a for a in range(dim)])
    return coef[cid]                                         # (M, d)


def assemble_level(dim: int, n: int, chunk: int = 1 << 20, coef: np.ndarray | None = None,
                   coef_cells: int = 0) -> Level:
    """Element-by-element P1 stiffness and vertex-rule weights (eq. 2.3, 2.6).

    S_ab = sum_K |K| grad(lam_a).A_K grad(lam_b);  w_a = sum_{K ni a} |K|/(d+1).
    A_K = I, or with `coef` (shape (coef_cells^d, d)) the diagonal SPD coefficient of eq. (2.1)
    that is constant on each cell of the coarsest mesh T_H (coef_cells = 1/H cells per side).
    Entries that cancel exactly in exact arithmetic (the diagonal couplings
    of these meshes) come out as round-off of size ~1e-17 |S_aa|; they are set
    to zero so that the sparsity is the true one.
    """
    h = 1.0 / n
    nodes, simp, _ = structured_mesh(dim, n)
    X = nodes.astype(np.float64) * h
    Nall = nodes.shape[0]
    rows, cols, vals = [], [], []
    wall = np.zeros(Nall)
    for s0 in range(0, simp.shape[0], chunk):
        sc = simp[s0:s0 + chunk]
        grads, vol = barycentric_gradients(X[sc])
        if coef is None:
            Ke = vol[:, None, None] * np.einsum("mad,mbd->mab", grads, grads)
        else:
            Ak = element_coefficients(coef, dim, coef_cells, X[sc])
            Ke = vol[:, None, None] * np.einsum("mad,md,mbd->mab", grads, Ak, grads)
        rows.append(np.repeat(sc, dim + 1, axis=1).ravel())
        cols.append(np.tile(sc, (1, dim + 1)).ravel())
        vals.append(Ke.ravel())
        np.add.at(wall, sc.ravel(), np.repeat(vol / (dim + 1), dim + 1))
    S = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(Nall, Nall))
    S.sum_duplicates()
    scale = np.abs(S.diagonal()).max()
    S.data[np.abs(S.data) <= 1e-12 * scale] = 0.0
    S.eliminate_zeros()
    inter = np.nonzero(interior_mask(nodes, n))[0]
    A = S[inter][:, inter].tocsr()
    lev = Level(dim=dim, n=n, h=h, nodes=nodes, interior=inter, A=A, w=wall[inter], S=S)
    _prepare_smoother(lev)
    return lev


def _prepare_smoother(lev: Level) -> None:
    """Red-black colouring by lattice parity (i+j[+l]) even = red."""
    lev.diag = lev.A.diagonal()
    lev.Aoff = (lev.A - sp.diags(lev.diag)).tocsr()
    par = lev.nodes[lev.interior].sum(axis=1) % 2
    lev.red = np.nonzero(par == 0)[0]
    lev.black = np.nonzero(par == 1)[0]
    lev.A_red = lev.Aoff[lev.red].tocsr()
    lev.A_black = lev.Aoff[lev.black].tocsr()


def same_colour_coupling(lev: Level) -> float:
    """Largest |a_ij| between distinct unknowns of the same colour (0 for a valid RB ordering)."""
    m = 0.0
    for idx in (lev.red, lev.black):
        sub = lev.Aoff[idx][:, idx]
        if sub.nnz:
            m = max(m, float(np.abs(sub.data).max()))
    return m


def prolongation(dim: int, n_coarse: int) -> sp.csr_matrix:
    """Matrix of the inclusion V_{2h} -> V_h (eq. 3.3) on the unknowns.

    Each fine node x is located in a coarse simplex (cell floor(x/H), then the
    simplex of that cell whose barycentric coordinates are all >= 0); row x of
    P holds the coarse basis functions' values lam_a(x) at the simplex's
    interior vertices.
    """
    n_f = 2 * n_coarse
    Hc = 1.0 / n_coarse
    cnodes, csimp, perms = structured_mesh(dim, n_coarse)
    fnodes, _, _ = structured_mesh(dim, n_f)
    fin = np.nonzero(interior_mask(fnodes, n_f))[0]
    cin_mask = interior_mask(cnodes, n_coarse)
    cpos = -np.ones(cnodes.shape[0], dtype=np.int64)
    cpos[cin_mask] = np.arange(int(cin_mask.sum()))
    x = fnodes[fin].astype(np.float64) / n_f            # physical coordinates
    cell = np.minimum(np.floor(x / Hc).astype(np.int64), n_coarse - 1)
    cell_id = cell @ np.array([n_coarse ** a for a in range(dim)])
    nper = len(perms)
    Xc = cnodes.astype(np.float64) * Hc
    chosen = -np.ones(fin.shape[0], dtype=np.int64)
    lam_chosen = np.zeros((fin.shape[0], dim + 1))
    for s in range(nper):
        sid = cell_id * nper + s
        V = Xc[csimp[sid]]                                 # (M, d+1, d)
        E = np.transpose(V[:, 1:, :] - V[:, :1, :], (0, 2, 1))
        lam_r = np.linalg.solve(E, (x - V[:, 0, :])[:, :, None])[:, :, 0]
        lam = np.concatenate([1.0 - lam_r.sum(axis=1, keepdims=True), lam_r], axis=1)
        ok = (chosen < 0) & np.all(lam >= -1e-12, axis=1)
        chosen[ok] = sid[ok]
        lam_chosen[ok] = lam[ok]
    assert np.all(chosen >= 0), "fine node outside every coarse simplex"
    cols = cpos[csimp[chosen]]                             # (M, d+1)
    rows = np.repeat(np.arange(fin.shape[0])[:, None], dim + 1, axis=1)
    keep = (cols >= 0) & (np.abs(lam_chosen) > 1e-14)
    P = sp.csr_matrix((lam_chosen[keep], (rows[keep], cols[keep])),
                      shape=(fin.shape[0], int(cin_mask.sum())))
    P.sum_duplicates()
    return P


# ---------------------------------------------------------------------------
# Hierarchy, smoother, V-cycle (Algorithm 3.1 step 1, eq. 3.4-3.5)
# ---------------------------------------------------------------------------


@dataclass
class Hierarchy:
    dim: int
    coarse_cells: int
    levels: list            # levels[0] is level 1 (= T_H)
    P_H: list = None        # P_H[k] = P_{H -> k} (level index k, 0-based)

    def level(self, k: int) -> Level:
        """1-based level access (level 1 is the coarse mesh)."""
        return self.levels[k - 1]


def build_hierarchy(dim: int, coarse_cells: int, refinements: int, coef: np.ndarray | None = None) -> Hierarchy:
    """Levels 1..refinements+1 of T_H (1/H = coarse_cells); coef: the diagonal coefficient per
    cell of T_H (see assemble_level), the same bilinear form on every level."""
    levs = []
    for k in range(refinements + 1):
        n = coarse_cells << k
        lev = assemble_level(dim, n, coef=coef, coef_cells=coarse_cells)
        if k > 0:
            lev.P = prolongation(dim, n // 2)
        levs.append(lev)
    levs[0].chol = sla.cho_factor(levs[0].A.toarray(), lower=True)
    hier = Hierarchy(dim=dim, coarse_cells=coarse_cells, levels=levs)
    # P_{H -> k} = P_k P_{k-1} ... P_2 (identity on level 1)
    PH = [sp.identity(levs[0].A.shape[0], format="csr")]
    for k in range(1, len(levs)):
        PH.append((levs[k].P @ PH[-1]).tocsr())
    hier.P_H = PH
    return hier


def rbgs_half(lev: Level, b: np.ndarray, u: np.ndarray, colour: str) -> None:
    """One colour of a Gauss-Seidel sweep: u_i <- (b_i - sum_{j!=i} a_ij u_j)/a_ii
    for every unknown i of that colour.  Unknowns of one colour do not couple,
    so updating them together is the sequential Gauss-Seidel update."""
    if colour == "red":
        idx, Ao = lev.red, lev.A_red
    else:
        idx, Ao = lev.black, lev.A_black
    u[idx] = (b[idx] - Ao @ u) / lev.diag[idx]


def smooth(lev: Level, b, u, sweeps: int, order: tuple) -> None:
    for _ in range(sweeps):
        for c in order:
            rbgs_half(lev, b, u, c)


# Chebyshev-Jacobi smoothing: the colour-free alternative smoother of the multigrid step.
# The smoothing polynomial is the Chebyshev polynomial of the Jacobi-preconditioned operator
# D^{-1} A shifted to the interval [lmin, lmax] = [lmax/ratio, lmax] of the high-frequency
# eigenvalues: after `degree` steps the error is p(D^{-1}A) e0 with
# p(lam) = T_degree((theta - lam)/delta) / T_degree(theta/delta), theta = (lmax+lmin)/2,
# delta = (lmax-lmin)/2, by the standard three-term Chebyshev iteration.  lmax = 2 bounds the
# spectrum of D^{-1}A for the 2d+1-point stiffness of these meshes (its eigenvalues are
# 1 - (cos + ... + cos)/d, all inside (0, 2)).
CHEB_LMAX = 2.0
CHEB_RATIO = 4.0


def chebyshev_smooth(lev: Level, b: np.ndarray, u: np.ndarray, degree: int,
                     lmax: float = CHEB_LMAX, ratio: float = CHEB_RATIO) -> None:
    """`degree` Chebyshev-Jacobi steps on A u = b, in place."""
    if degree <= 0:
        return
    lmin = lmax / ratio
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sig = theta / delta
    rho = 1.0 / sig
    d = (b - lev.A @ u) / lev.diag / theta
    u += d
    for _ in range(1, degree):
        r = (b - lev.A @ u) / lev.diag
        rho_new = 1.0 / (2.0 * sig - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
        u += d


def vcycle(hier: Hierarchy, k: int, b: np.ndarray, u: np.ndarray,
           nu_pre: int = 2, nu_post: int = 2, smoother: str = "rbgs") -> np.ndarray:
    """One V(nu_pre, nu_post) cycle for A_k u = b from the initial guess u.  smoother:
    "rbgs" (red-black Gauss-Seidel sweeps) or "chebyshev" (Chebyshev-Jacobi steps of degree
    nu_pre / nu_post)."""
    lev = hier.level(k)
    u = u.copy()
    if k == 1:
        return sla.cho_solve(lev.chol, b)
    if smoother == "chebyshev":
        chebyshev_smooth(lev, b, u, nu_pre)
    else:
        smooth(lev, b, u, nu_pre, ("red", "black"))
    r = b - lev.A @ u
    bc = lev.P.T @ r
    ec = vcycle(hier, k - 1, bc, np.zeros_like(bc), nu_pre, nu_post, smoother)
    u += lev.P @ ec
    if smoother == "chebyshev":
        chebyshev_smooth(lev, b, u, nu_post)
    else:
        smooth(lev, b, u, nu_post, ("black", "red"))
    return u


# ---------------------------------------------------------------------------
# Discrete nonlinear problem (2.7) with vertex quadrature
# ---------------------------------------------------------------------------


def load_vector(lev: Level, g_nodal_level: np.ndarray) -> np.ndarray:
    """(g, phi_i) by the vertex rule: w_i g(x_i) on the unknowns."""
    return lev.w * g_nodal_level.ravel()[lev.interior]


def restrict_nodal(g_fine: np.ndarray, dim: int, n_fine: int, n: int) -> np.ndarray:
    """Nodal values of g on the coarser lattice (every (n_fine/n)-th node)."""
    s = n_fine // n
    g = g_fine.reshape((n_fine + 1,) * dim)
    sl = tuple(slice(None, None, s) for _ in range(dim))
    return np.ascontiguousarray(g[sl])


def nonlinear_residual(lev, G, kind, a, U):
    return lev.A @ U + lev.w * f_val(kind, a, U) - G


def newton_full(lev: Level, G, kind, a, U0=None, tol=1e-13, maxit=60, direct="sparse"):
    """Newton's method on A U + W f(U) = G (the discrete problem 2.7).

    Jacobian A + W diag(f'(U)) is SPD for monotone f; stops when
    ||delta||_inf <= tol * max(1, ||U||_inf).  Returns (U, iterations)."""
    U = np.zeros(lev.A.shape[0]) if U0 is None else U0.copy()
    for it in range(1, maxit + 1):
        R = nonlinear_residual(lev, G, kind, a, U)
        J = lev.A + sp.diags(lev.w * f_der(kind, a, U))
        if direct == "dense":
            delta = -sla.cho_solve(sla.cho_factor(J.toarray(), lower=True), R)
        else:
            delta = -spla.spsolve(J.tocsc(), R)
        U = U + delta
        if np.max(np.abs(delta)) <= tol * max(1.0, np.max(np.abs(U))):
            return U, it
    raise RuntimeError("Newton on the full discrete problem did not converge")


# ---------------------------------------------------------------------------
# Algorithm 3.1: one correction step
# ---------------------------------------------------------------------------


@dataclass
class StepInfo:
    newton_iters: int = 0
    alpha: float = 1.0
    c: np.ndarray = None
    u_tilde: np.ndarray = None
    dropped_u_tilde: bool = False


def augmented_newton(lev: Level, PHk: sp.csr_matrix, ut: np.ndarray, G: np.ndarray, kind: str, a: float,
                     tol: float = 1e-6, maxit: int = 30):
    """Newton on (3.6): find y = (c, alpha) with u = P_{H->k} c + alpha u~ such that
    B^T A_k B y + B^T W f(B y) = B^T G,  B = [P_{H->k} | u~].

    The (N_H+1) Galerkin matrix is assembled from its blocks
    [[P^T A P, P^T A u~], [u~^T A P, u~^T A u~]]; P^T A_k P is the coarse
    stiffness A_H (checked separately).  Start (c, alpha) = (0, 1), stop on
    ||delta||_inf <= tol*max(1, ||y||_inf)."""
    NH = PHk.shape[1]
    B = sp.hstack([PHk, sp.csr_matrix(ut[:, None])]).tocsr()
    AB = lev.A @ B
    Kaug = (B.T @ AB).toarray()
    Gaug = B.T @ G
    y = np.zeros(NH + 1)
    y[-1] = 1.0
    for it in range(1, maxit + 1):
        U = B @ y
        R = Kaug @ y + B.T @ (lev.w * f_val(kind, a, U)) - Gaug
        D = sp.diags(lev.w * f_der(kind, a, U))
        J = Kaug + (B.T @ (D @ B)).toarray()
        delta = -sla.cho_solve(sla.cho_factor(J, lower=True), R)
        y = y + delta
        if np.max(np.abs(delta)) <= tol * max(1.0, np.max(np.abs(y))):
            return y, B, it
    raise RuntimeError("augmented Newton did not converge")


def augmented_chord(lev: Level, PHk: sp.csr_matrix, ut: np.ndarray, G: np.ndarray, kind: str, a: float,
                    tol: float = 1e-6, maxit: int = 30):
    """The chord (simplified Newton) iteration on (3.6): Newton's step with the Jacobian of the
    first iterate, assembled and factored once.  Its fixed point is Newton's (the residual is
    the same); only the rate differs, linear instead of quadratic.  Same start (c, alpha) =
    (0, 1) and stopping rule as augmented_newton.  This is the reading the mixed-precision
    GPU path takes for the nonlinear solver the paper leaves open."""
    NH = PHk.shape[1]
    B = sp.hstack([PHk, sp.csr_matrix(ut[:, None])]).tocsr()
    Kaug = (B.T @ (lev.A @ B)).toarray()
    Gaug = B.T @ G
    y = np.zeros(NH + 1)
    y[-1] = 1.0
    fac = None
    for it in range(1, maxit + 1):
        U = B @ y
        R = Kaug @ y + B.T @ (lev.w * f_val(kind, a, U)) - Gaug
        if fac is None:
            D = sp.diags(lev.w * f_der(kind, a, U))
            fac = sla.cho_factor(Kaug + (B.T @ (D @ B)).toarray(), lower=True)
        delta = -sla.cho_solve(fac, R)
        y = y + delta
        if np.max(np.abs(delta)) <= tol * max(1.0, np.max(np.abs(y))):
            return y, B, it
    raise RuntimeError("augmented chord iteration did not converge")


def augmented_fixed_point(lev: Level, PHk: sp.csr_matrix, ut: np.ndarray, G: np.ndarray, kind: str, a: float,
                          tol: float = 1e-6, maxit: int = 60):
    """The fixed-point iteration on (3.6), the other nonlinear solver the paper names: the
    linear part implicit, the nonlinear term at the previous iterate,
    B^T A_k B y_{k+1} = B^T G - B^T W f(B y_k),  B = [P_{H->k} | u~],
    from (c, alpha) = (0, 1), with Newton's stopping rule.  It converges when the nonlinear
    term is a contraction relative to the Galerkin stiffness (mild nonlinearities)."""
    NH = PHk.shape[1]
    B = sp.hstack([PHk, sp.csr_matrix(ut[:, None])]).tocsr()
    Kaug = (B.T @ (lev.A @ B)).toarray()
    Gaug = B.T @ G
    fac = sla.cho_factor(Kaug, lower=True)
    y = np.zeros(NH + 1)
    y[-1] = 1.0
    for it in range(1, maxit + 1):
        y_new = sla.cho_solve(fac, Gaug - B.T @ (lev.w * f_val(kind, a, B @ y)))
        delta = y_new - y
        y = y_new
        if np.max(np.abs(delta)) <= tol * max(1.0, np.max(np.abs(y))):
            return y, B, it
    raise RuntimeError("augmented fixed-point iteration did not converge")


def correction_step(hier: Hierarchy, k: int, u: np.ndarray, G: np.ndarray, kind: str, a: float,
                    m: int = 2, nu_pre: int = 2, nu_post: int = 2, tol: float = 1e-6,
                    smoother: str = "rbgs", nonlinear: str = "newton"):
    """u^{(l+1)} = SemilinearMG(V_H, u^{(l)}, V_{h_k}) (Algorithm 3.1)."""
    lev = hier.level(k)
    # step 1 (eq. 3.4): a(u^, v) = (g, v) - (f(x, u^{(l)}), v)
    b = G - lev.w * f_val(kind, a, u)
    ut = u.copy()
    for _ in range(m):                     # eq. (3.5): m multigrid steps from u^{(l)}
        ut = vcycle(hier, k, b, ut, nu_pre, nu_post, smoother)
    # step 2 (eq. 3.6): semilinear problem on V_H + span{u~}
    solve = {"newton": augmented_newton, "chord": augmented_chord, "fixed_point": augmented_fixed_point}[nonlinear]
    y, B, iters = solve(lev, hier.P_H[k - 1], ut, G, kind, a, tol)
    info = StepInfo(newton_iters=iters, alpha=float(y[-1]), c=y[:-1].copy(), u_tilde=ut)
    return B @ y, info


# ---------------------------------------------------------------------------
# Algorithm 3.2: full multigrid
# ---------------------------------------------------------------------------


@dataclass
class FMGResult:
    u: list                       # u[k-1] = u_{h_k} on the unknowns of level k
    steps: list                   # StepInfo per (level, correction)
    level1_iters: int = 0


def fmg(hier: Hierarchy, g_fine: np.ndarray, kind: str, a: float, m: int = 2, p: int = 1,
        nu_pre: int = 2, nu_post: int = 2, tol: float = 1e-6, tol_level1: float = 1e-6,
        keep_levels: bool = True, smoother: str = "rbgs", nonlinear: str = "newton") -> FMGResult:
    n_levels = len(hier.levels)
    n_fine = hier.levels[-1].n
    dim = hier.dim
    lev1 = hier.level(1)
    G1 = load_vector(lev1, restrict_nodal(g_fine, dim, n_fine, lev1.n))
    # step 1: the semilinear problem on V_{h_1} solved exactly (Newton, dense)
    u, it1 = newton_full(lev1, G1, kind, a, tol=tol_level1, direct="dense")
    us = [u]
    steps = []
    for k in range(2, n_levels + 1):
        lev = hier.level(k)
        G = load_vector(lev, restrict_nodal(g_fine, dim, n_fine, lev.n))
        u = lev.P @ u                      # u^{(0)}_{h_k} = u_{h_{k-1}} (natural inclusion)
        for _ in range(p):
            u, info = correction_step(hier, k, u, G, kind, a, m, nu_pre, nu_post, tol, smoother, nonlinear)
            steps.append((k, info))
        if keep_levels:
            us.append(u)
        else:
            us = [u]
    return FMGResult(u=us, steps=steps, level1_iters=it1)


# ---------------------------------------------------------------------------
# Norms and errors
# ---------------------------------------------------------------------------


def to_nodal(lev: Level, U: np.ndarray) -> np.ndarray:
    """Unknowns -> full (n+1)^d nodal array with zero boundary, x fastest."""
    full = np.zeros(lev.nodes.shape[0])
    full[lev.interior] = U
    return full.reshape((lev.n + 1,) * lev.dim)


def from_nodal(lev: Level, arr: np.ndarray) -> np.ndarray:
    return np.asarray(arr).ravel()[lev.interior]


def discrete_l2(lev: Level, e: np.ndarray) -> float:
    return float(math.sqrt(lev.h ** lev.dim * np.sum(e * e)))


def energy_norm(lev: Level, e: np.ndarray) -> float:
    return float(math.sqrt(max(e @ (lev.A @ e), 0.0)))


_QUAD = {
    # degree-2 rules on the reference simplex, barycentric points and weights (sum 1)
    2: (np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]]), np.full(3, 1.0 / 3.0)),
    3: (np.array([[0.5854101966249685, 0.1381966011250105, 0.1381966011250105, 0.1381966011250105],
                  [0.1381966011250105, 0.5854101966249685, 0.1381966011250105, 0.1381966011250105],
                  [0.1381966011250105, 0.1381966011250105, 0.5854101966249685, 0.1381966011250105],
                  [0.1381966011250105, 0.1381966011250105, 0.1381966011250105, 0.5854101966249685]]),
        np.full(4, 0.25)),
}


def fe_errors(lev: Level, U: np.ndarray, problem) -> tuple[float, float]:
    """L2 and H1-seminorm errors of the P1 function U against the exact u*,
    integrated element by element with a degree-2 rule."""
    dim = lev.dim
    nodes, simp, _ = structured_mesh(dim, lev.n)
    X = nodes.astype(np.float64) * lev.h
    full = np.zeros(nodes.shape[0])
    full[lev.interior] = U
    bary, wq = _QUAD[dim]
    l2 = 0.0
    h1 = 0.0
    for s0 in range(0, simp.shape[0], 1 << 18):
        sc = simp[s0:s0 + (1 << 18)]
        V = X[sc]
        grads, vol = barycentric_gradients(V)
        gradU = np.einsum("ma,mad->md", full[sc], grads)
        for q in range(bary.shape[0]):
            pts = np.einsum("a,mad->md", bary[q], V)
            uq = full[sc] @ bary[q]
            us, gs = problem.grad_u_star(pts)
            l2 += float(np.sum(wq[q] * vol * (us - uq) ** 2))
            h1 += float(np.sum(wq[q] * vol * np.sum((gs - gradU) ** 2, axis=1)))
    return math.sqrt(l2), math.sqrt(h1)

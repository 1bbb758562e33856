// Nonlinear and dense steps of the full multigrid method:
//   * level-1 setup: the dense inverse of A_1 for the exact coarsest solve of the cycles;
//   * Algorithm 3.2 step 1: the semilinear problem on V_{h_1} solved exactly by Newton;
//   * Algorithm 3.1 step 2 (eq. 3.6): the semilinear problem on V_{H,h_k} = V_H + span{u~},
//     solved by Newton on y = (c, alpha), u = P_{H->k} c + alpha u~.  Every Newton iteration
//     assembles the (N_H+1)-dimensional system from one pass over the fine nodes (the
//     O(N_k) assembly the paper's work estimate, Theorem 3.3, counts per nonlinear step).
//
// Galerkin structure of the augmented system with B = [P_{H->k} | u~] and vertex quadrature
// (weights w = h_k^d):
//   R_H   = A_H c + alpha t + P^T (w f(U)) - G_H            t = P^T A_k u~,  G_H = P^T (w g)
//   R_a   = t.c + alpha s + u~.(w f(U)) - gamma             s = u~.A_k u~,   gamma = u~.(w g)
//   J_HH  = A_H + P^T diag(w f'(U)) P,  J_Ha = t + P^T (w f'(U) u~),  J_aa = s + u~.(w f'(U) u~)
// with U = alpha u~ + P c and A_H = P^T A_k P the coarse stiffness (nested P1 spaces).
//
// P_{H->k} c at a fine node x is the P1 interpolant of the coarse nodal values: x lies in
// coarse cell floor(x / s) (s = 2^(k-1) fine cells per coarse cell) with local offsets o in
// [0, s)^d; sorting the axes by decreasing o gives the Kuhn simplex v_0 = 0,
// v_{t+1} = v_t + e_{pi_t} and barycentric weights lambda_0 = (s - o_{pi_0})/s,
// lambda_t = (o_{pi_{t-1}} - o_{pi_t})/s, lambda_d = o_{pi_{d-1}}/s.
//
// Reductions are deterministic: per-thread accumulators in shared memory, fixed-order
// warp-shuffle and block sums, fixed-order sums over blocks and coarse cells.
#include <cuda_runtime.h>

#include "fmg_internal.cuh"

namespace fmg {

namespace {

// ------------------------------------------------------------------ dense SPD solve (one CTA)
// In-place Cholesky (lower) of the n x n matrix M (row-major, leading dimension ld, in shared
// memory) followed by the solve M x = rhs (rhs overwritten).  `shared` must hold 2 doubles.
// If `drop_last` and the last pivot is below drop_tol times its original value, the last
// unknown is frozen (its increment is 0) and *dropped is set.  Returns false if not SPD.
__device__ bool block_chol_solve(double* M, int n, int ld, double* rhs, double* shared, bool drop_last,
                                 double drop_tol, int* dropped) {
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  __shared__ int bad;
  __shared__ int drop;
  if (tid == 0) {
    bad = 0;
    drop = 0;
    shared[1] = drop_last ? M[(long long)(n - 1) * ld + (n - 1)] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double d = M[k * ld + k];
      if (drop_last && k == n - 1 && !(d > drop_tol * shared[1])) {
        drop = 1;
        d = 1.0;
        for (int j = 0; j < k; ++j) M[k * ld + j] = 0.0;
        rhs[k] = 0.0;
      } else if (!(d > 0.0)) {
        bad = 1;
        d = 1.0;
      }
      const double r = sqrt(d);
      M[k * ld + k] = r;
      shared[0] = 1.0 / r;
    }
    __syncthreads();
    const double inv = shared[0];
    for (int i = k + 1 + tid; i < n; i += nt) M[i * ld + k] *= inv;
    __syncthreads();
    const int m = n - k - 1;
    for (int idx = tid; idx < m * m; idx += nt) {
      const int i = k + 1 + idx / m;
      const int j = k + 1 + idx % m;
      if (j <= i) M[i * ld + j] -= M[i * ld + k] * M[j * ld + k];
    }
    __syncthreads();
  }
  // forward substitution L y = rhs
  for (int k = 0; k < n; ++k) {
    if (tid == 0) rhs[k] /= M[k * ld + k];
    __syncthreads();
    const double yk = rhs[k];
    for (int i = k + 1 + tid; i < n; i += nt) rhs[i] -= M[i * ld + k] * yk;
    __syncthreads();
  }
  // back substitution L^T x = y
  for (int k = n - 1; k >= 0; --k) {
    if (tid == 0) rhs[k] /= M[k * ld + k];
    __syncthreads();
    const double xk = rhs[k];
    for (int i = tid; i < k; i += nt) rhs[i] -= M[k * ld + i] * xk;
    __syncthreads();
  }
  if (dropped) *dropped = drop;
  return bad == 0;
}

// Level-1 unknown r <-> nodal offset of interior node (r % m + 1, (r/m) % m + 1, r/m^2 + 1).
__device__ __forceinline__ long long node_of(int r, int m, int dim) {
  const long long np = m + 2;
  const int i = r % m + 1;
  const int j = (r / m) % m + 1;
  if (dim == 2) return (long long)j * np + i;
  const int l = r / (m * m) + 1;
  return ((long long)l * np + j) * np + i;
}

// A_1 entry between unknowns p and q: sigma (2d on the diagonal, -1 for axis neighbours).
__device__ __forceinline__ double stiff_entry(int p, int q, int m, int dim, double sigma) {
  if (p == q) return sigma * 2 * dim;
  int pc[3] = {p % m, (p / m) % m, p / (m * m)};
  int qc[3] = {q % m, (q / m) % m, q / (m * m)};
  int dist = 0;
  for (int a = 0; a < dim; ++a) dist += abs(pc[a] - qc[a]);
  return dist == 1 ? -sigma : 0.0;
}

__global__ void k_coarse_inverse(int dim, int n1, double* __restrict__ Ainv, DevState* st) {
  extern __shared__ double sm[];
  const int m = n1 - 1;
  const int N = dim == 2 ? m * m : m * m * m;
  const int ld = N + 1;
  double* M = sm;
  double* rhs = M + (size_t)N * ld;
  double* sh = rhs + N;
  const double sigma = dim == 2 ? 1.0 : 1.0 / n1;
  for (int col = 0; col < N; ++col) {
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int i = idx / N, j = idx % N;
      M[i * ld + j] = stiff_entry(i, j, m, dim, sigma);
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) rhs[i] = (i == col) ? 1.0 : 0.0;
    __syncthreads();
    bool ok = block_chol_solve(M, N, ld, rhs, sh, false, 0.0, nullptr);
    if (!ok && threadIdx.x == 0) atomicOr(&st->flags, kFlagNotSPD);
    for (int i = threadIdx.x; i < N; i += blockDim.x) Ainv[(long long)i * N + col] = rhs[i];
    __syncthreads();
  }
}

// Algorithm 3.2 step 1: Newton on A_1 U + w f(U) = w g, from U = 0.
__global__ void k_level1_newton(int dim, int n1, const double* __restrict__ g, double* __restrict__ u, int kind,
                                double a, double tol, int maxit, DevState* st) {
  extern __shared__ double sm[];
  const int m = n1 - 1;
  const int N = dim == 2 ? m * m : m * m * m;
  const int ld = N + 1;
  double* M = sm;
  double* rhs = M + (size_t)N * ld;
  double* U = rhs + N;
  double* Fp = U + N;
  double* sh = Fp + N;
  __shared__ int done;
  __shared__ double red[2];
  const double h = 1.0 / n1;
  const double sigma = dim == 2 ? 1.0 : h;
  const double w = dim == 2 ? h * h : h * h * h;
  for (int i = threadIdx.x; i < N; i += blockDim.x) U[i] = 0.0;
  if (threadIdx.x == 0) done = 0;
  __syncthreads();
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    // residual R = A U + w f(U) - w g  (stored negated in rhs) and Jacobian
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      double F, D;
      f_eval<double>(kind, a, U[p], F, D);
      double au = 0.0;
      for (int q = 0; q < N; ++q) au += stiff_entry(p, q, m, dim, sigma) * U[q];
      rhs[p] = -(au + w * F - w * g[node_of(p, m, dim)]);
      Fp[p] = w * D;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int i = idx / N, j = idx % N;
      M[i * ld + j] = stiff_entry(i, j, m, dim, sigma) + (i == j ? Fp[i] : 0.0);
    }
    __syncthreads();
    const bool ok = block_chol_solve(M, N, ld, rhs, sh, false, 0.0, nullptr);
    if (threadIdx.x == 0) {
      double dmax = 0.0, umax = 0.0;
      bool finite = true;
      for (int p = 0; p < N; ++p) {
        const double v = U[p] + rhs[p];
        if (!isfinite(v)) finite = false;
        dmax = fmax(dmax, fabs(rhs[p]));
        umax = fmax(umax, fabs(v));
      }
      red[0] = dmax;
      red[1] = umax;
      if (!ok) atomicOr(&st->flags, kFlagNotSPD);
      if (!finite) atomicOr(&st->flags, kFlagNonfinite);
      if (!ok || !finite) done = 2;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < N; p += blockDim.x) U[p] += rhs[p];
    __syncthreads();
    if (threadIdx.x == 0 && done == 0 && red[0] <= tol * fmax(1.0, red[1])) done = 1;
    __syncthreads();
    if (done) break;
  }
  if (threadIdx.x == 0) {
    if (done != 1) atomicOr(&st->flags, kFlagNewtonCap);
    st->level1_iters = it > maxit ? maxit : it;
  }
  for (int p = threadIdx.x; p < N; p += blockDim.x) u[node_of(p, m, dim)] = U[p];
}

// ------------------------------------------------------------------ augmented problem
template <int D>
struct Aug {
  static constexpr int NV = 1 << D;                      // vertices of a coarse cell
  static constexpr int NP = NV * (NV + 1) / 2;           // vertex pairs (packed upper)
  static constexpr int VA = 0;                           // vector channel A
  static constexpr int VB = NV;                          // vector channel B
  static constexpr int PP = 2 * NV;                      // pair channel
  static constexpr int S0 = 2 * NV + NP;                 // scalar channels
  static constexpr int NVAL = 2 * NV + NP + 2;
  static constexpr int NT = D == 2 ? 256 : 128;          // threads per block
};

__device__ __forceinline__ int pair_index(int NV, int v, int u) {
  if (v > u) {
    const int t = v;
    v = u;
    u = t;
  }
  return v * NV - (v * (v - 1)) / 2 + (u - v);
}

struct AugArgs {
  int dim, nc, s, n, kind, maxit, level_index, bpc;
  double a, w, sigma_k, sigma_H, tol;
  double* u;            // u~ on entry, u^{(l+1)} on exit (level-k nodal)
  const double* g;      // level-k nodal g
  double* partials;     // [cells * bpc][NVAL]
  double* c;            // coarse nodal iterate ((nc+1)^d, boundary 0)
  double* sys;          // t[NH] G_H[NH] s gamma
  DevState* st;
};

// Bounded grid barrier for the cooperative launch (all blocks co-resident).  On timeout the
// abort word is set and every block leaves at its next check.
__device__ void grid_barrier(DevState* st, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* genp = &st->bar_gen;
    const unsigned gen = *genp;
    __threadfence();
    const unsigned arrived = atomicAdd(&st->bar_count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*genp == gen) {
        __nanosleep(64);
        if (++spins > (1ll << 25)) {
          atomicOr(&st->flags, kFlagTimeout);
          atomicExch(&st->abort, 1);
          break;
        }
        if (((volatile int*)&st->abort)[0]) break;
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Kuhn simplex of the local offsets o (in [0,s)^D): vertex ids and barycentric numerators.
template <int D>
__device__ __forceinline__ void kuhn_simplex(const int* o, int s, int* vid, int* lnum) {
  int pi[D];
#pragma unroll
  for (int q = 0; q < D; ++q) pi[q] = q;
  // sort axes by decreasing offset (ties keep axis order)
#pragma unroll
  for (int q = 0; q < D; ++q)
#pragma unroll
    for (int r = 0; r < D - 1 - q; ++r)
      if (o[pi[r]] < o[pi[r + 1]]) {
        const int t = pi[r];
        pi[r] = pi[r + 1];
        pi[r + 1] = t;
      }
  vid[0] = 0;
  lnum[0] = s - o[pi[0]];
#pragma unroll
  for (int q = 1; q < D; ++q) {
    vid[q] = vid[q - 1] | (1 << pi[q - 1]);
    lnum[q] = o[pi[q - 1]] - o[pi[q]];
  }
  vid[D] = (1 << D) - 1;
  lnum[D] = o[pi[D - 1]];
}

// Coarse nodal offset of vertex v of cell (I,J,L).
__device__ __forceinline__ long long cell_vertex_node(int D, const int* cellc, int v, int nc) {
  const long long cp = nc + 1;
  long long off = 0, mul = 1;
  for (int q = 0; q < D; ++q) {
    off += (long long)(cellc[q] + ((v >> q) & 1)) * mul;
    mul *= cp;
  }
  return off;
}

// Phase kinds of the per-node pass.
enum { kPre = 0, kNewton = 1, kUpdate = 2 };

template <int D>
__device__ void node_pass(const AugArgs& A, int phase, double* acc, const double* cv, double alpha, int cell,
                          int bic) {
  using G = Aug<D>;
  const int tid = threadIdx.x;
  const int s = A.s;
  const long long np = A.n + 1;
  int cellc[3] = {0, 0, 0};
  {
    int t = cell;
    for (int q = 0; q < D; ++q) {
      cellc[q] = t % A.nc;
      t /= A.nc;
    }
  }
  const long long per_cell = ipow(s, D);
  const double inv_s = 1.0 / s;
  const long long stride = (long long)A.bpc * G::NT;
  for (long long li = (long long)bic * G::NT + tid; li < per_cell; li += stride) {
    int o[D];
    long long t = li;
    long long off = 0, mul = 1;
    bool interior = true;
#pragma unroll
    for (int q = 0; q < D; ++q) {
      o[q] = (int)(t % s);
      t /= s;
      const int x = cellc[q] * s + o[q];
      if (x == 0) interior = false;
      off += (long long)x * mul;
      mul *= np;
    }
    if (!interior) continue;
    int vid[D + 1], lnum[D + 1];
    kuhn_simplex<D>(o, s, vid, lnum);
    double lam[D + 1];
#pragma unroll
    for (int q = 0; q <= D; ++q) lam[q] = lnum[q] * inv_s;
    const double ut = A.u[off];
    if (phase == kPre) {
      double au;
      if (D == 2) {
        au = 4.0 * ut - ((A.u[off - 1] + A.u[off + 1]) + (A.u[off - np] + A.u[off + np]));
      } else {
        const long long pl = np * np;
        au = A.sigma_k *
             (6.0 * ut - (((A.u[off - 1] + A.u[off + 1]) + (A.u[off - np] + A.u[off + np])) +
                          (A.u[off - pl] + A.u[off + pl])));
      }
      const double wg = A.w * A.g[off];
#pragma unroll
      for (int q = 0; q <= D; ++q) {
        acc[(G::VA + vid[q]) * G::NT + tid] += au * lam[q];
        acc[(G::VB + vid[q]) * G::NT + tid] += wg * lam[q];
      }
      acc[(G::S0) * G::NT + tid] += ut * au;
      acc[(G::S0 + 1) * G::NT + tid] += wg * ut;
    } else {
      double U = alpha * ut;
#pragma unroll
      for (int q = 0; q <= D; ++q) U += lam[q] * cv[vid[q]];
      if (phase == kUpdate) {
        A.u[off] = U;
        continue;
      }
      double F, Fp;
      f_eval<double>(A.kind, A.a, U, F, Fp);
      const double q_ = A.w * F;
      const double d_ = A.w * Fp;
      const double du = d_ * ut;
#pragma unroll
      for (int q = 0; q <= D; ++q) {
        acc[(G::VA + vid[q]) * G::NT + tid] += q_ * lam[q];
        acc[(G::VB + vid[q]) * G::NT + tid] += du * lam[q];
        const double dl = d_ * lam[q];
#pragma unroll
        for (int r = q; r <= D; ++r) acc[(G::PP + pair_index(G::NV, vid[q], vid[r])) * G::NT + tid] += dl * lam[r];
      }
      acc[(G::S0) * G::NT + tid] += q_ * ut;
      acc[(G::S0 + 1) * G::NT + tid] += du * ut;
    }
  }
}

// Block sum of the accumulator rows into partials[blockIdx.x][*] (fixed order).
template <int D>
__device__ void block_reduce_rows(const double* acc, double* out) {
  using G = Aug<D>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = G::NT / 32;
  __syncthreads();
  for (int v = warp; v < G::NVAL; v += nw) {
    double x = 0.0;
    for (int t = lane; t < G::NT; t += 32) x += acc[v * G::NT + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) out[v] = x;
  }
  __syncthreads();
}

// Sum over the blocks of each cell, then over the cells around each coarse node (fixed
// orders).  Result: per coarse unknown p: vecA[p], vecB[p]; per unknown pair: pairs; scalars.
// Writes into the dense system arrays of block 0 in shared memory.
template <int D>
__device__ void gather_cells(const AugArgs& A, double* cellsum) {
  using G = Aug<D>;
  const int ncell = (int)ipow(A.nc, D);
  for (int idx = threadIdx.x; idx < ncell * G::NVAL; idx += blockDim.x) {
    const int cell = idx / G::NVAL, v = idx % G::NVAL;
    double x = 0.0;
    for (int b = 0; b < A.bpc; ++b) x += __ldcg(&A.partials[((long long)cell * A.bpc + b) * G::NVAL + v]);
    cellsum[idx] = x;
  }
  __syncthreads();
}

// Coordinates of coarse unknown p.
template <int D>
__device__ __forceinline__ void unknown_coords(int p, int nc, int* z) {
  const int m = nc - 1;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    z[q] = p % m + 1;
    p /= m;
  }
}

// Sum of channel `ch` at vertex p over the 2^D cells around coarse node p.
template <int D>
__device__ double node_channel(const double* cellsum, int nc, const int* z, int ch) {
  using G = Aug<D>;
  double x = 0.0;
  for (int o = 0; o < G::NV; ++o) {
    int cc[3];
    bool ok = true;
    int cell = 0, mul = 1;
    for (int q = 0; q < D; ++q) {
      cc[q] = z[q] - ((o >> q) & 1);
      if (cc[q] < 0 || cc[q] >= nc) ok = false;
      cell += cc[q] * mul;
      mul *= nc;
    }
    if (!ok) continue;
    x += cellsum[(long long)cell * G::NVAL + ch + o];
  }
  return x;
}

template <int D>
__device__ double pair_channel(const double* cellsum, int nc, const int* zp, const int* zq) {
  using G = Aug<D>;
  double x = 0.0;
  for (int o = 0; o < G::NV; ++o) {
    int cc[3];
    bool ok = true;
    int cell = 0, mul = 1, vq = 0;
    for (int q = 0; q < D; ++q) {
      cc[q] = zp[q] - ((o >> q) & 1);
      if (cc[q] < 0 || cc[q] >= nc) ok = false;
      const int dq = zq[q] - cc[q];
      if (dq < 0 || dq > 1) ok = false;
      vq |= dq << q;
      cell += cc[q] * mul;
      mul *= nc;
    }
    if (!ok) continue;
    x += cellsum[(long long)cell * G::NVAL + G::PP + pair_index(G::NV, o, vq)];
  }
  return x;
}

template <int D>
__global__ void __launch_bounds__(Aug<D>::NT) k_augmented(AugArgs A) {
  using G = Aug<D>;
  extern __shared__ double sm[];
  double* acc = sm;                                 // NVAL * NT
  __shared__ double cv[G::NV];
  __shared__ double alpha_sh;
  __shared__ int stop;
  const int tid = threadIdx.x;
  const unsigned nblocks = gridDim.x;
  const int cell = blockIdx.x / A.bpc;
  const int bic = blockIdx.x % A.bpc;
  const int ncell = (int)ipow(A.nc, D);
  const int NH = (int)ipow(A.nc - 1, D);
  const int NA = NH + 1;
  int cellc[3] = {0, 0, 0};
  {
    int t = cell;
    for (int q = 0; q < D; ++q) {
      cellc[q] = t % A.nc;
      t /= A.nc;
    }
  }
  // block-0 scratch (after acc): cellsum [ncell * NVAL], M [NA * (NA+1)], R [NA], misc
  double* cellsum = acc + G::NVAL * G::NT;
  double* M = cellsum + (size_t)ncell * G::NVAL;
  double* R = M + (size_t)NA * (NA + 1);
  double* sh = R + NA;
  double* t_vec = A.sys;
  double* gh_vec = A.sys + NH;
  double* s_gam = A.sys + 2 * NH;

  // -------- phase 0: t = P^T A_k u~, G_H = P^T (w g), s, gamma
  for (int v = 0; v < G::NVAL; ++v) acc[v * G::NT + tid] = 0.0;
  node_pass<D>(A, kPre, acc, nullptr, 0.0, cell, bic);
  block_reduce_rows<D>(acc, A.partials + (long long)blockIdx.x * G::NVAL);
  grid_barrier(A.st, nblocks);
  if (blockIdx.x == 0) {
    gather_cells<D>(A, cellsum);
    for (int p = tid; p < NH; p += blockDim.x) {
      int z[3];
      unknown_coords<D>(p, A.nc, z);
      t_vec[p] = node_channel<D>(cellsum, A.nc, z, G::VA);
      gh_vec[p] = node_channel<D>(cellsum, A.nc, z, G::VB);
    }
    if (tid == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int c = 0; c < ncell; ++c) {
        s0 += cellsum[(long long)c * G::NVAL + G::S0];
        s1 += cellsum[(long long)c * G::NVAL + G::S0 + 1];
      }
      s_gam[0] = s0;
      s_gam[1] = s1;
      A.st->alpha_cur = 1.0;
      A.st->converged = 0;
    }
    const long long cn = ipow(A.nc + 1, D);
    for (long long i = tid; i < cn; i += blockDim.x) A.c[i] = 0.0;
  }
  grid_barrier(A.st, nblocks);

  // -------- Newton iterations
  int it = 0;
  for (it = 1; it <= A.maxit; ++it) {
    if (tid < G::NV) cv[tid] = __ldcg(&A.c[cell_vertex_node(D, cellc, tid, A.nc)]);
    if (tid == 0) {
      alpha_sh = ((volatile double*)&A.st->alpha_cur)[0];
      stop = ((volatile int*)&A.st->abort)[0];
    }
    for (int v = 0; v < G::NVAL; ++v) acc[v * G::NT + tid] = 0.0;
    __syncthreads();
    if (stop) break;
    node_pass<D>(A, kNewton, acc, cv, alpha_sh, cell, bic);
    block_reduce_rows<D>(acc, A.partials + (long long)blockIdx.x * G::NVAL);
    grid_barrier(A.st, nblocks);
    if (blockIdx.x == 0) {
      gather_cells<D>(A, cellsum);
      const double alpha = alpha_sh;
      const double sig = A.sigma_H;
      // residual (negated into R) and Jacobian
      for (int p = tid; p < NH; p += blockDim.x) {
        int z[3];
        unknown_coords<D>(p, A.nc, z);
        // A_H c at p
        const long long cp = A.nc + 1;
        long long off = 0, mul = 1;
        for (int q = 0; q < D; ++q) {
          off += (long long)z[q] * mul;
          mul *= cp;
        }
        double nb = 0.0;
        mul = 1;
        for (int q = 0; q < D; ++q) {
          nb += __ldcg(&A.c[off - mul]) + __ldcg(&A.c[off + mul]);
          mul *= cp;
        }
        const double ahc = sig * (2.0 * D * __ldcg(&A.c[off]) - nb);
        const double rp = ahc + alpha * t_vec[p] + node_channel<D>(cellsum, A.nc, z, G::VA) - gh_vec[p];
        R[p] = -rp;
        M[(long long)p * (NA + 1) + NH] = t_vec[p] + node_channel<D>(cellsum, A.nc, z, G::VB);
        for (int q2 = 0; q2 < NH; ++q2) {
          int zq[3];
          unknown_coords<D>(q2, A.nc, zq);
          int dist = 0;
          bool near = true;
          for (int q = 0; q < D; ++q) {
            const int dd = zq[q] - z[q];
            dist += abs(dd);
            if (dd < -1 || dd > 1) near = false;
          }
          double v = 0.0;
          if (near) {
            v = pair_channel<D>(cellsum, A.nc, z, zq);
            if (dist == 0) v += sig * 2.0 * D;
            else if (dist == 1) v -= sig;
          }
          M[(long long)p * (NA + 1) + q2] = v;
        }
      }
      if (tid == 0) {
        double s2 = 0.0, s3 = 0.0, tc = 0.0;
        for (int c = 0; c < ncell; ++c) {
          s2 += cellsum[(long long)c * G::NVAL + G::S0];
          s3 += cellsum[(long long)c * G::NVAL + G::S0 + 1];
        }
        for (int p = 0; p < NH; ++p) {
          int z[3];
          unknown_coords<D>(p, A.nc, z);
          const long long cp = A.nc + 1;
          long long off = 0, mul = 1;
          for (int q = 0; q < D; ++q) {
            off += (long long)z[q] * mul;
            mul *= cp;
          }
          tc += t_vec[p] * __ldcg(&A.c[off]);
        }
        R[NH] = -(tc + alpha * s_gam[0] + s2 - s_gam[1]);
        M[(long long)NH * (NA + 1) + NH] = s_gam[0] + s3;
      }
      __syncthreads();
      for (int p = tid; p < NH; p += blockDim.x) M[(long long)NH * (NA + 1) + p] = M[(long long)p * (NA + 1) + NH];
      __syncthreads();
      int dropped = 0;
      const bool ok = block_chol_solve(M, NA, NA + 1, R, sh, true, 1e-14, &dropped);
      if (tid == 0) {
        double dmax = 0.0, ymax = 0.0;
        bool finite = true;
        const long long cp = A.nc + 1;
        for (int p = 0; p < NH; ++p) {
          int z[3];
          unknown_coords<D>(p, A.nc, z);
          long long off = 0, mul = 1;
          for (int q = 0; q < D; ++q) {
            off += (long long)z[q] * mul;
            mul *= cp;
          }
          const double nv = __ldcg(&A.c[off]) + R[p];
          if (!isfinite(nv)) finite = false;
          A.c[off] = nv;
          dmax = fmax(dmax, fabs(R[p]));
          ymax = fmax(ymax, fabs(nv));
        }
        const double na = alpha + R[NH];
        if (!isfinite(na)) finite = false;
        dmax = fmax(dmax, fabs(R[NH]));
        ymax = fmax(ymax, fabs(na));
        A.st->alpha_cur = na;
        if (dropped) atomicOr(&A.st->flags, kFlagDropped);
        if (!ok) atomicOr(&A.st->flags, kFlagNotSPD);
        if (!finite) atomicOr(&A.st->flags, kFlagNonfinite);
        if (!ok || !finite) A.st->abort = 1;
        if (dmax <= A.tol * fmax(1.0, ymax)) A.st->converged = 1;
        __threadfence();
      }
    }
    grid_barrier(A.st, nblocks);
    if (tid == 0) stop = ((volatile int*)&A.st->converged)[0] | ((volatile int*)&A.st->abort)[0];
    __syncthreads();
    if (stop) break;
  }
  if (blockIdx.x == 0 && tid == 0) {
    const int conv = ((volatile int*)&A.st->converged)[0];
    if (!conv) atomicOr(&A.st->flags, kFlagNewtonCap);
    A.st->newton_iters[A.level_index] += it > A.maxit ? A.maxit : it;
    A.st->alpha[A.level_index] = ((volatile double*)&A.st->alpha_cur)[0];
  }
  // -------- final update u = alpha u~ + P_{H->k} c
  if (tid < G::NV) cv[tid] = __ldcg(&A.c[cell_vertex_node(D, cellc, tid, A.nc)]);
  if (tid == 0) alpha_sh = ((volatile double*)&A.st->alpha_cur)[0];
  __syncthreads();
  node_pass<D>(A, kUpdate, acc, cv, alpha_sh, cell, bic);
}

template <int D>
size_t aug_smem(int nc) {
  using G = Aug<D>;
  const int ncell = (int)ipow(nc, D);
  const int NA = (int)ipow(nc - 1, D) + 1;
  return sizeof(double) * ((size_t)G::NVAL * G::NT + (size_t)ncell * G::NVAL + (size_t)NA * (NA + 1) + NA + 4);
}

}  // namespace

// ============================================================================ launchers

cudaError_t launch_coarse_inverse(int dim, LevelGeo g1, double* Ainv, DevState* st, cudaStream_t s) {
  const int m = g1.n - 1;
  const int N = (int)ipow(m, dim);
  const size_t smem = sizeof(double) * ((size_t)N * (N + 1) + N + 4);
  cudaError_t e = cudaFuncSetAttribute(k_coarse_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_coarse_inverse<<<1, 256, smem, s>>>(dim, g1.n, Ainv, st);
  return cudaGetLastError();
}

cudaError_t launch_level1_newton(int dim, LevelGeo g1, const double* gn, double* u, int kind, double a, double tol,
                                 int maxit, DevState* st, cudaStream_t s) {
  const int m = g1.n - 1;
  const int N = (int)ipow(m, dim);
  const size_t smem = sizeof(double) * ((size_t)N * (N + 1) + 3 * (size_t)N + 4);
  cudaError_t e = cudaFuncSetAttribute(k_level1_newton, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_level1_newton<<<1, 256, smem, s>>>(dim, g1.n, gn, u, kind, a, tol, maxit, st);
  return cudaGetLastError();
}

int aug_nvals(int dim) { return dim == 2 ? Aug<2>::NVAL : Aug<3>::NVAL; }

// Blocks per coarse cell for the cooperative launch; at most what fits co-resident.
static int aug_bpc(int dim, int coarse_cells, int num_sms, size_t* smem_out, int* nt_out) {
  const int ncell = (int)ipow(coarse_cells, dim);
  int occ = 0;
  size_t smem;
  int nt;
  if (dim == 2) {
    smem = aug_smem<2>(coarse_cells);
    nt = Aug<2>::NT;
    cudaFuncSetAttribute(k_augmented<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_augmented<2>, nt, smem);
  } else {
    smem = aug_smem<3>(coarse_cells);
    nt = Aug<3>::NT;
    cudaFuncSetAttribute(k_augmented<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_augmented<3>, nt, smem);
  }
  if (smem_out) *smem_out = smem;
  if (nt_out) *nt_out = nt;
  const int maxblocks = occ * num_sms;
  int bpc = maxblocks / ncell;
  if (bpc < 1) bpc = 0;  // cannot launch: not enough co-resident blocks
  return bpc;
}

void aug_configure(int dim, int coarse_cells, AugBuffers* ab) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    sms = 0;
  size_t smem = 0;
  int nt = 0;
  const int bpc = sms > 0 ? aug_bpc(dim, coarse_cells, sms, &smem, &nt) : 1;
  ab->bpc = bpc;
  ab->smem = smem;
  ab->nt = nt;
  ab->partial_items = (size_t)ipow(coarse_cells, dim) * (bpc > 0 ? bpc : 1);
}

cudaError_t launch_augmented(int dim, int coarse_cells, int level, LevelGeo gk, double* u, const double* gn,
                             int kind, double a, double tol, int maxit, const AugBuffers& ab, DevState* st,
                             int level_index, cudaStream_t s) {
  const size_t smem = ab.smem;
  const int nt = ab.nt;
  const int bpc = ab.bpc;
  if (bpc < 1 || nt < 1) return cudaErrorInvalidConfiguration;
  const int ncell = (int)ipow(coarse_cells, dim);
  if ((size_t)ncell * bpc > ab.partial_items) return cudaErrorInvalidValue;
  AugArgs A;
  A.dim = dim;
  A.nc = coarse_cells;
  A.s = 1 << (level - 1);
  A.n = gk.n;
  A.kind = kind;
  A.maxit = maxit;
  A.level_index = level_index;
  A.bpc = bpc;
  A.a = a;
  const double h = 1.0 / gk.n;
  A.w = dim == 2 ? h * h : h * h * h;
  A.sigma_k = dim == 2 ? 1.0 : h;
  A.sigma_H = dim == 2 ? 1.0 : 1.0 / coarse_cells;
  A.tol = tol;
  A.u = u;
  A.g = gn;
  A.partials = ab.partials;
  A.c = ab.c;
  A.sys = ab.sys;
  A.st = st;
  // barrier words and abort/converged flags start cleared
  cudaError_t e = cudaMemsetAsync(&st->bar_count, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncell * bpc);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (dim == 2) return cudaLaunchKernelEx(&cfg, k_augmented<2>, A);
  return cudaLaunchKernelEx(&cfg, k_augmented<3>, A);
}

}  // namespace fmg

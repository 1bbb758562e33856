// Nonlinear and dense steps of the full multigrid method:
//   * level-1 setup: the dense inverse of A_1 for the exact coarsest solve of the cycles;
//   * Algorithm 3.2 step 1: the semilinear problem on V_{h_1} solved exactly by Newton;
//   * Algorithm 3.1 step 2 (eq. 3.6): the semilinear problem on V_{H,h_k} = V_H + span{u~},
//     solved by Newton on y = (c, alpha), u = P_{H->k} c + alpha u~.  Every Newton iteration
//     assembles the (N_H+1)-dimensional system from one pass over the fine nodes (the
//     O(N_k) assembly the work estimate of Theorem 3.3 counts per nonlinear step).
//
// Galerkin structure of the augmented system with B = [P_{H->k} | u~] and vertex quadrature
// (weights w = h_k^d):
//   R_H   = A_H c + alpha t + P^T (w f(U)) - G_H            t = P^T A_k u~,  G_H = P^T (w g)
//   R_a   = t.c + alpha s + u~.(w f(U)) - gamma             s = u~.A_k u~,   gamma = u~.(w g)
//   J_HH  = A_H + P^T diag(w f'(U)) P,  J_Ha = t + P^T (w f'(U) u~),  J_aa = s + u~.(w f'(U) u~)
// with U = alpha u~ + P c and A_H = P^T A_k P the coarse stiffness (nested P1 spaces).
//
// P_{H->k} c at a fine node is the P1 interpolant of the coarse nodal values.  A fine node
// lies in coarse cell floor(x/s) (s = 2^(k-1) fine cells per coarse cell) at local offsets
// o in [0,s)^d; sorting the axes by decreasing offset (ties: lower axis first) gives the Kuhn
// simplex v_0 = 0, v_{t+1} = v_t + e_{pi_t}, with barycentric weights
// lambda_0 = (s - o_{pi_0})/s, lambda_t = (o_{pi_{t-1}} - o_{pi_t})/s, lambda_d = o_{pi_{d-1}}/s.
//
// Fine pass layout.  A thread walks a column of a coarse cell: all offsets fixed except the
// last one (z).  Along the column the simplex changes only where z crosses the fixed
// offsets, so the column splits into d segments; on a segment every lambda_t is affine in z,
// lambda_t = (P_t + R_t z)/s, and every sum the system needs is a combination of the
// segment's moments sum X, sum X z, sum X z^2.  The thread accumulates those moments in
// registers (FP64 for the residual; FP32 or FP64 for the Jacobian) and converts them to the
// cell's vertex channels once per segment.  The residual sums carry f(U) - g, so G_H and gamma
// are never formed apart; the first pass also gathers t and s
// (at (c, alpha) = (0, 1), U = u~), so no separate precompute pass is needed.
//
// Reductions are deterministic: per-thread channel rows in shared memory, fixed-order block
// sums, fixed-order sums over blocks and cells.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "fmg_ff.cuh"
#include "fmg_internal.cuh"
#include "fmg_phase.cuh"

namespace fmg {

namespace {

// ------------------------------------------------------------------ small dense SPD solve
// 1/d for d > 0 from the fast FP32 reciprocal estimate (about 2 ulp), refined by Newton's
// iteration for 1/d (y <- y (2 - d y)) in the target precision: one step for FP32, two for
// FP64 (the error squares each step).
__device__ __forceinline__ float recip_pivot(float d) {
  const float y = __fdividef(1.0f, d);
  return y * (2.0f - d * y);
}
__device__ __forceinline__ double recip_pivot(double d) {
  double y = (double)__fdividef(1.0f, (float)d);
  y = y * (2.0 - d * y);
  return y * (2.0 - d * y);
}

// LDL^T factorization (no pivoting), on ONE warp, of the n x n SPD matrix A whose leading
// nb = n - border unknowns are banded (A_ij = 0 for i, j < nb and |i - j| > band) and whose
// last row and column (border = 1) or none (border = 0) are dense: the coarse Jacobians of
// the Newton steps in lexicographic order (band m or m^2 for the level-1 stencil; m + 1 or
// m^2 + m + 1 for the coarse-simplex couplings of the augmented system, whose alpha unknown
// is the border).  Row-major, leading dimension ld, shared memory, precision T; only the
// lower triangle is read, and its entries outside the pattern must be zero.  Eliminating
// unknown k touches only the rows R_k = {k+1 .. min(k+band, nb-1)} and the border row, so
// the pattern is closed under the elimination and step k updates the lower triangle of
// R_k x R_k -- at most q(q+1)/2 entries, q = band + border -- instead of the whole trailing
// triangle.  Each entry gets the same operations in the same order as in a dense
// elimination (the skipped updates subtract exact zeros), so the factor is the dense one.
// In place: below the diagonal A[i][k] keeps the k-th column of the reduced matrix
// (= L_ik d_k), and rd[k] = 1/d_k.
//
// The positions (a, c), c <= a < q, of R_k x R_k are dealt to the lanes once (NS slots per
// lane).  A position moves along the diagonal with k (band rows: stride ld + 1) or along the
// border row (stride 1), so each lane keeps, per slot, the offsets of its entry and of the two
// column-k entries it needs plus their strides; a slot whose entry has left the matrix keeps
// the offsets of its last update and stops storing.  At most four slots per lane:
// (band + border)(band + border + 1) / 2 <= 128.  The step is branch-free (predicated
// stores; every lane forms a reciprocal and the one that updated the next pivot keeps it),
// so it costs a few loads, one update and a store per slot, the pivot's reciprocal and one
// __syncwarp.  If
// drop_last and the last pivot (the Schur complement of the last unknown) falls below drop_tol
// times the original last diagonal entry, rd[n-1] = 0: that unknown is frozen (*dropped = 1).
// Returns false if a pivot is not positive.
template <typename T, int NS, int FN = 0, int FBAND = 0>
__device__ bool ldlt_band_warp_ns(T* A, int n_arg, int ld_arg, T* rd, int band_arg, int border, bool drop_last,
                                  double drop_tol, int* dropped) {
  // FN, FBAND > 0: the size and band fixed at compile time (ld = FN + 1), which folds the
  // offsets and strides into constants
  const int n = FN > 0 ? FN : n_arg;
  const int ld = FN > 0 ? FN + 1 : ld_arg;
  const int band = FBAND > 0 ? FBAND : band_arg;
  const int lane = threadIdx.x & 31;
  const int nb = n - border;
  const int q = band + border;
  const int P = q * (q + 1) / 2;
  int oij[NS], oik[NS], ojk[NS];   // offsets at step k
  int sij[NS], sik[NS], sjk[NS];   // their strides per step
  int kend[NS];                    // the entry is updated for k < kend
  int piv[NS];                     // 1: band pivot, 2: border pivot
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int t = lane + 32 * s;
    int a = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= t) ++a;
    while (a * (a + 1) / 2 > t) --a;
    const int c = t - a * (a + 1) / 2;
    kend[s] = 0;
    piv[s] = 0;
    oij[s] = oik[s] = ojk[s] = 0;
    sij[s] = sik[s] = sjk[s] = 0;
    if (t >= P) continue;
    if (a < band) {   // band rows k+1+a, k+1+c
      kend[s] = nb - 1 - a;
      oij[s] = (1 + a) * ld + 1 + c;
      oik[s] = (1 + a) * ld;
      ojk[s] = (1 + c) * ld;
      sij[s] = sik[s] = sjk[s] = ld + 1;
      piv[s] = (a == 0) ? 1 : 0;
    } else if (c < band) {   // border row nb, band column k+1+c
      kend[s] = nb - 1 - c;
      oij[s] = nb * ld + 1 + c;
      oik[s] = nb * ld;
      ojk[s] = (1 + c) * ld;
      sij[s] = 1;
      sik[s] = 1;
      sjk[s] = ld + 1;
    } else {   // the border pivot (nb, nb)
      kend[s] = nb;
      oij[s] = nb * ld + nb;
      oik[s] = ojk[s] = nb * ld;
      sik[s] = sjk[s] = 1;
      piv[s] = 2;
    }
    if (kend[s] <= 0) {   // never updated (the band is wider than the matrix): a safe address
      oij[s] = oik[s] = ojk[s] = 0;
      sij[s] = sik[s] = sjk[s] = 0;
    }
  }
  const T last0 = drop_last ? A[(n - 1) * ld + (n - 1)] : T(0);
  const T drop_at = T(drop_tol) * last0;
  bool bad = false, drop = false;
  // reciprocal of pivot k (0 with the flag when it is dropped or not positive)
  auto pivot_recip = [&](int k, T d, bool& isdrop, bool& isbad) -> T {
    isdrop = drop_last && k == n - 1 && !(d > drop_at);
    isbad = !isdrop && !(d > T(0));
    return (isdrop || isbad) ? T(0) : recip_pivot(d);
  };
  {
    bool dd, bb;
    const T r0 = pivot_recip(0, A[0], dd, bb);
    if (lane == 0) {
      rd[0] = r0;
      drop = dd;
      bad = bb;
    }
  }
  __syncwarp();
#pragma unroll 2
  for (int k = 0; k + 1 < n; ++k) {
    const T r = rd[k];
    T pv = T(1);
    bool own = false;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const bool act = k < kend[s];
      const T v = A[oij[s]] - A[oik[s]] * r * A[ojk[s]];
      if (act) A[oij[s]] = v;
      const bool isp = act && (piv[s] == 1 || (piv[s] == 2 && k == nb - 1));
      pv = isp ? v : pv;
      own = own || isp;
      // advance only while the next step still updates the entry, so that the offsets never
      // leave the matrix (the loads above run for finished slots too)
      const bool nxt = k + 1 < kend[s];
      oij[s] += nxt ? sij[s] : 0;
      oik[s] += nxt ? sik[s] : 0;
      ojk[s] += nxt ? sjk[s] : 0;
    }
    bool dd, bb;
    const T rn = pivot_recip(k + 1, pv, dd, bb);
    if (own) {
      rd[k + 1] = rn;
      drop = drop || dd;
      bad = bad || bb;
    }
    __syncwarp();
  }
  if (dropped) *dropped = __any_sync(0xffffffffu, drop) ? 1 : 0;
  return !__any_sync(0xffffffffu, bad);
}

// Dispatch on the slots per lane the pattern needs; false if it needs more than four.
template <typename T>
__device__ bool ldlt_band_warp(T* A, int n, int ld, T* rd, int band, int border, bool drop_last, double drop_tol,
                               int* dropped) {
  if (border < 0 || border > 1) return false;
  const int q = band + border;
  const int ns = (q * (q + 1) / 2 + 31) >> 5;
  switch (ns) {
    case 0:
    case 1: return ldlt_band_warp_ns<T, 1>(A, n, ld, rd, band, border, drop_last, drop_tol, dropped);
    case 2: return ldlt_band_warp_ns<T, 2>(A, n, ld, rd, band, border, drop_last, drop_tol, dropped);
    case 3: return ldlt_band_warp_ns<T, 3>(A, n, ld, rd, band, border, drop_last, drop_tol, dropped);
    case 4: return ldlt_band_warp_ns<T, 4>(A, n, ld, rd, band, border, drop_last, drop_tol, dropped);
    default: return false;
  }
}

// Solves L D L^T x = b with the factor of ldlt_band_warp (same n, band, border), on one warp
// (lane l holds entries l and l + 32; n <= 64).  Forward substitution column by column over
// the band rows (one shuffle per step; the rows of the half that the band does not reach are
// skipped by warp-uniform tests), the border row's part as one dot product after it; then the
// backward substitution row by row, the border unknown first and its contribution to every
// other row in one parallel step.  b (FP64, shared) is overwritten by x.  Only the calling
// warp takes part; the caller synchronizes before others read b.
template <typename T>
__device__ void ldlt_solve_band_warp(const T* A, int n, int ld, const T* rd, int band, int border, double* b) {
  const int lane = threadIdx.x & 31;
  const int nb = n - border;
  const int i0 = lane, i1 = lane + 32;
  T z0 = i0 < n ? (T)b[i0] : T(0), z1 = i1 < n ? (T)b[i1] : T(0);
  // forward: w_k = z_k / d_k, then z_i -= A_ik w_k for band rows k < i <= min(k + band, nb - 1)
  for (int k = 0; k < nb; ++k) {
    const T zk = __shfl_sync(0xffffffffu, k < 32 ? z0 : z1, k & 31);
    const T wk = zk * rd[k];
    const int hi = min(k + band, nb - 1);
    if (k + 1 < 32 && i0 > k && i0 <= hi) z0 -= A[i0 * ld + k] * wk;
    if (hi >= 32 && i1 > k && i1 <= hi) z1 -= A[i1 * ld + k] * wk;
    if (i0 == k) z0 = wk;
    if (i1 == k) z1 = wk;
  }
  // the border row: z_nb -= sum_k A_{nb,k} w_k, then w_nb = z_nb / d_nb
  if (border) {
    T part = T(0);
    if (i0 < nb) part += A[nb * ld + i0] * z0;
    if (i1 < nb) part += A[nb * ld + i1] * z1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (i0 == nb) z0 = (z0 - part) * rd[nb];
    if (i1 == nb) z1 = (z1 - part) * rd[nb];
  }
  // backward: x_k = w_k - (1/d_k) sum_{i>k} A_ik x_i; s holds the running sums
  T s0 = T(0), s1 = T(0);
  if (border) {
    const T xb = __shfl_sync(0xffffffffu, nb < 32 ? z0 : z1, nb & 31);
    if (i0 < nb) s0 = A[nb * ld + i0] * xb;
    if (i1 < nb) s1 = A[nb * ld + i1] * xb;
  }
  for (int k = nb - 1; k >= 0; --k) {
    T xk = T(0);
    if (i0 == k) xk = z0 - rd[k] * s0;
    if (i1 == k) xk = z1 - rd[k] * s1;
    xk = __shfl_sync(0xffffffffu, xk, k & 31);
    if (i0 == k) z0 = xk;
    if (i1 == k) z1 = xk;
    const int lo = k - band;
    if (lo < 32 && i0 < k && i0 >= lo) s0 += A[k * ld + i0] * xk;
    if (k > 32 && i1 < k && i1 >= lo) s1 += A[k * ld + i1] * xk;
  }
  if (i0 < n) b[i0] = (double)z0;
  if (i1 < n) b[i1] = (double)z1;
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

// The 2d edge weights at level-1 unknown p (interior node of T_H, order as node_of): the
// coefficient's weights at level shift 0 (every cell of T_H is a coefficient cell).
__device__ __forceinline__ void level1_weights(const VarCoef& vc, int p, int m, int dim, double* w) {
  const int i = p % m + 1, j = (p / m) % m + 1, l = dim == 3 ? p / (m * m) + 1 : 0;
  if (dim == 2)
    edge_weights_t<2, double>(vc, 0, i, j, l, w);
  else
    edge_weights_t<3, double>(vc, 0, i, j, l, w);
}

// Entry (p, q) of the level-1 stiffness A_1: sigma times the sum of p's edge weights on the
// diagonal, minus sigma times the weight of their common edge for axis neighbours, zero
// otherwise (A = I: every weight 1, i.e. 2d sigma and -sigma).
__device__ double level1_entry(int p, int q, int m, int dim, double sigma, const VarCoef& vc) {
  int dist = 0, axis = 0, dir = 0;
  int pp = p, qq = q;
  for (int a = 0; a < dim; ++a) {
    const int d = qq % m - pp % m;
    if (d != 0) {
      axis = a;
      dir = d;
    }
    dist += abs(d);
    pp /= m;
    qq /= m;
  }
  if (dist > 1) return 0.0;
  if (!vc.a64) return dist == 0 ? sigma * 2 * dim : -sigma;
  double w[6];
  level1_weights(vc, p, m, dim, w);
  if (dist == 1) return -sigma * w[2 * axis + (dir > 0 ? 1 : 0)];
  double sw = 0.0;
  for (int e = 0; e < 2 * dim; ++e) sw += w[e];
  return sigma * sw;
}

// Writes the dense A_1 into M.
__device__ void fill_stiffness(double* M, int N, int ld, int m, int dim, double sigma, const VarCoef& vc) {
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int p = idx / N, q = idx % N;
    M[p * ld + q] = level1_entry(p, q, m, dim, sigma, vc);
  }
}

// Level-1 setup: LDL^T of A_1 once, then A_1^{-1} column by column (one thread per column).
// Launched with 64 threads.
__global__ void k_coarse_inverse(int dim, int n1, double* __restrict__ Ainv, DevState* st, VarCoef vc) {
  pdl_start();
  extern __shared__ double sm[];
  const int m = n1 - 1;
  const int N = dim == 2 ? m * m : m * m * m;
  const int ld = N + 1;
  double* M = sm;
  double* rd = M + (size_t)N * ld;
  const double sigma = dim == 2 ? 1.0 : 1.0 / n1;
  fill_stiffness(M, N, ld, m, dim, sigma, vc);
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool ok = ldlt_band_warp<double>(M, N, ld, rd, dim == 2 ? m : m * m, 0, false, 0.0, nullptr);
    if (!ok && threadIdx.x == 0) atomicOr(&st->flags, kFlagNotSPD);
  }
  __syncthreads();
  // column `col` of the inverse: L D L^T x = e_col (A^{-1} is symmetric: column = row), with
  // L_kj = M[k][j] / d_j below the diagonal
  for (int col = threadIdx.x; col < N; col += blockDim.x) {
    double* x = Ainv + (long long)col * N;
    for (int k = 0; k < N; ++k) {
      double acc = (k == col) ? 1.0 : 0.0;
      for (int j = 0; j < k; ++j) acc -= M[k * ld + j] * rd[j] * x[j];
      x[k] = acc;
    }
    for (int k = 0; k < N; ++k) x[k] *= rd[k];
    for (int k = N - 1; k >= 0; --k) {
      double acc = 0.0;
      for (int j = k + 1; j < N; ++j) acc += M[j * ld + k] * x[j];
      x[k] -= rd[k] * acc;
    }
  }
}

// Algorithm 3.2 step 1: Newton on A_1 U + w f(U) = w g, from U = 0 (one CTA).  The residual,
// the iterate and the convergence test are FP64; the Jacobian A_1 + diag(w f'(U)) is factored
// in precision T (T = float in the mixed path: an inexact Newton step whose error the next
// FP64 residual corrects, so the iteration converges to the same FP64 solution).
template <typename T>
__device__ __forceinline__ void k_level1_newton_body(int dim, int n1, const double* __restrict__ g, double* __restrict__ u, int kind,
                                double a, double tol, int maxit, DevState* st, int out_ff, VarCoef vc) {
  extern __shared__ double sm[];
  const int m = n1 - 1;
  const int N = dim == 2 ? m * m : m * m * m;
  const int ld = N + 1;
  double* U = sm;
  double* rhs = U + N;
  double* Fp = rhs + N;
  T* L = reinterpret_cast<T*>(Fp + N);
  T* work = L + (size_t)N * ld;
  T* invd = work + N;
  __shared__ int done, ok_sh;
  const double h = 1.0 / n1;
  const double sigma = dim == 2 ? 1.0 : h;
  const double w = dim == 2 ? h * h : h * h * h;
  const int band = dim == 2 ? m : m * m;   // lexicographic half-bandwidth of the 2d+1-point stencil
  for (int i = threadIdx.x; i < N; i += blockDim.x) U[i] = 0.0;
  // entries outside the band are zero and the factorization never writes them
  for (int i = threadIdx.x; i < N * ld; i += blockDim.x) L[i] = T(0);
  if (threadIdx.x == 0) done = 0;
  __syncthreads();
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      double F, D;
      f_eval<double>(kind, a, U[p], F, D);
      // (A U)_p from the stencil: sigma (2d U_p - sum of interior axis neighbours), or with
      // the coefficient sigma sum_e w_e (U_p - U_e) (boundary neighbours are zero)
      double au;
      if (vc.a64) {
        double wt[6];
        level1_weights(vc, p, m, dim, wt);
        double acc = 0.0;
        int rem = p, mul = 1;
        for (int ax = 0; ax < dim; ++ax) {
          const int c = rem % m;
          rem /= m;
          acc += wt[2 * ax] * (U[p] - (c > 0 ? U[p - mul] : 0.0));
          acc += wt[2 * ax + 1] * (U[p] - (c < m - 1 ? U[p + mul] : 0.0));
          mul *= m;
        }
        au = sigma * acc;
      } else {
        double nb = 0.0;
        int rem = p, mul = 1;
        for (int ax = 0; ax < dim; ++ax) {
          const int c = rem % m;
          rem /= m;
          if (c > 0) nb += U[p - mul];
          if (c < m - 1) nb += U[p + mul];
          mul *= m;
        }
        au = sigma * (2.0 * dim * U[p] - nb);
      }
      rhs[p] = -(au + w * F - w * g[node_of(p, m, dim)]);
      Fp[p] = w * D;
    }
    __syncthreads();
    // the lower band of the Jacobian A_1 + diag(w f'(U)) (the factor of the previous
    // iteration overwrote it)
    for (int idx = threadIdx.x; idx < N * (band + 1); idx += blockDim.x) {
      const int p = idx / (band + 1), q = p - idx % (band + 1);
      if (q < 0) continue;
      const double v = level1_entry(p, q, m, dim, sigma, vc) + (p == q ? Fp[p] : 0.0);
      L[p * ld + q] = (T)v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // the benchmark shapes (2D 1/H = 8, 3D 1/H = 4) with their size and band fixed at compile time
      const bool okw = (dim == 2 && N == 49 && band == 7)
                           ? ldlt_band_warp_ns<T, 1, 49, 7>(L, N, ld, invd, band, 0, false, 0.0, nullptr)
                       : (dim == 3 && N == 27 && band == 9)
                           ? ldlt_band_warp_ns<T, 2, 27, 9>(L, N, ld, invd, band, 0, false, 0.0, nullptr)
                           : ldlt_band_warp<T>(L, N, ld, invd, band, 0, false, 0.0, nullptr);
      ldlt_solve_band_warp<T>(L, N, ld, invd, band, 0, rhs);
      if (threadIdx.x == 0) ok_sh = okw ? 1 : 0;
    }
    __syncthreads();
    const bool ok = ok_sh != 0;
    if (threadIdx.x < 32) {
      double dmax = 0.0, umax = 0.0;
      bool finite = true;
      for (int p = threadIdx.x; p < N; p += 32) {
        const double v = U[p] + rhs[p];
        if (!isfinite(v)) finite = false;
        dmax = fmax(dmax, fabs(rhs[p]));
        umax = fmax(umax, fabs(v));
        U[p] = v;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        umax = fmax(umax, __shfl_xor_sync(0xffffffffu, umax, o));
      }
      finite = __all_sync(0xffffffffu, finite);
      if (threadIdx.x == 0) {
        if (!ok) atomicOr(&st->flags, kFlagNotSPD);
        if (!finite) atomicOr(&st->flags, kFlagNonfinite);
        if (!ok || !finite) done = 2;
        else if (dmax <= tol * fmax(1.0, umax)) done = 1;
      }
    }
    __syncthreads();
    if (done) break;
  }
  if (threadIdx.x == 0) {
    if (done != 1) atomicOr(&st->flags, kFlagNewtonCap);
    st->level1_iters = it > maxit ? maxit : it;
  }
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    if (out_ff)
      ff_store(u + node_of(p, m, dim), ff_from_double(U[p]));
    else
      u[node_of(p, m, dim)] = U[p];
  }
}

template <typename T>
__global__ void k_level1_newton(int dim, int n1, const double* __restrict__ g, double* __restrict__ u, int kind,
                                double a, double tol, int maxit, DevState* st, int out_ff, VarCoef vc) { pdl_start(); k_level1_newton_body<T>(dim, n1, g, u, kind, a, tol, maxit, st, out_ff, vc); }

// ------------------------------------------------------------------ augmented problem
template <int D, bool JF32>
struct Aug {
  static constexpr int NV = 1 << D;             // vertices of a coarse cell
  static constexpr int NP = NV * (NV + 1) / 2;  // vertex pairs (packed upper)
  // channel layout of a block's partial sums (all stored as double)
  // f(U) and g enter the residual only as f(U) - g (R_H = A_H c + alpha t + P^T w (f(U) - g),
  // R_a = t.c + alpha s + u~.w (f(U) - g)), so G_H and gamma need no channels of their own
  static constexpr int RA = 0;                  // sum w (f(U) - g) lambda_v        [NV]
  static constexpr int SA = NV;                 // sum w (f(U) - g) u~               [1]
  static constexpr int TT = NV + 1;             // sum (A u~) lambda_v  (first pass) [NV]
  static constexpr int SS = 2 * NV + 1;         // sum u~ A u~          (first pass) [1]
  static constexpr int JB = 2 * NV + 2;         // sum w f'(U) u~ lambda_v           [NV]
  static constexpr int JP = 3 * NV + 2;         // sum w f'(U) lambda_v lambda_u     [NP]
  static constexpr int JS = 3 * NV + 2 + NP;    // sum w f'(U) u~^2                  [1]
  static constexpr int NVAL = 3 * NV + 3 + NP;
  static constexpr int NT = D == 2 ? 256 : 128;
};

// Channel rows of a block: one row of NT per-thread partial sums per channel.  FP64 path:
// every channel FP64, already scaled by its quadrature weight.  Mixed path: the residual
// channels (RA .. SS) are float-float pairs (hi, lo) in their 8-byte slots and carry no weight
// (RA is scaled by w/s, SA by w, TT by 1/s when the block sum is converted to FP64), so a pass
// does no FP64 arithmetic; the Jacobian channels (JB .. JS) are FP32 rows after them (FP32
// products to begin with), which halves their shared memory.
template <int D, bool JF32>
struct Rows {
  using G = Aug<D, JF32>;
  static constexpr int NF = JF32 ? G::NVAL - G::JB : 0;   // FP32 rows
  static constexpr int ND = G::NVAL - NF;                  // FP64 rows
  static constexpr size_t bytes = (size_t)ND * G::NT * sizeof(double) + (size_t)NF * G::NT * sizeof(float);
  __device__ static float* jac(double* acc) { return reinterpret_cast<float*>(acc + (size_t)ND * G::NT); }
  __device__ static const float* jac(const double* acc) {
    return reinterpret_cast<const float*>(acc + (size_t)ND * G::NT);
  }
  // zero this thread's rows of the channels the pass fills
  __device__ static void zero(double* acc, bool first, bool fixed_point, int tid) {
    if ((JF32 || fixed_point) && !first) {
      for (int v = 0; v <= G::SA; ++v) acc[v * G::NT + tid] = 0.0;
      return;
    }
    const int nd = fixed_point ? G::JB : ND;   // no Jacobian channels in the fixed-point iteration
    for (int v = 0; v < nd; ++v) acc[v * G::NT + tid] = 0.0;
    if (fixed_point) return;
    float* f = jac(acc);
    for (int v = 0; v < NF; ++v) f[v * G::NT + tid] = 0.f;
  }
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
  int dim, nc, s, ls, n, kind, maxit, level_index, bpc, chunk;   // s = 2^ls fine cells per coarse cell
  int fixed_point;      // 1: fixed-point iteration (Galerkin stiffness only, no Jacobian)
  int out_f64;          // mixed path: the update writes u as FP64 (the solve's result) instead of float-float
  int split_update;     // 1: the final update is left to k_aug_update (block 0 writes c and alpha to cfin)
  double a, w, sigma_k, sigma_H, tol;
  ff a_ff, sigma_ff;    // mixed path: a and sigma_k as float-float
  double* u;            // u~ on entry, u^{(l+1)} on exit (level-k nodal; float-float in the mixed path)
  const double* g;      // level-k nodal g (float-float in the mixed path)
  double* partials;     // two buffers of [cells * bpc][NVAL] block partial rows
  long long pstride;    // doubles per buffer
  const double* Ainv;   // A_H^{-1} (= A_1^{-1}, h_1 = H), dense NH x NH, preconditioner
  DevState* st;
  double* cfin;         // [(nc+1)^d] c, then alpha (split_update)
  long long bar_spins;  // polls of the grid barrier before it times out
  int bar_skip;         // test hook: this block skips its first barrier arrival (-1: none)
  VarCoef vc;           // the coefficient A(x) (vc.a64 == nullptr: A = I)
  const int* jtab;      // mixed path: the Jacobian gather table (k_aug_jtab)
};

// Bounded grid barrier for the cooperative launch (all blocks co-resident).  A waiting block
// gives up after `spins` polls: the timeout flag and the abort word are set and every block
// leaves at its next check.  skip (the failure-detection test hook): this block does not
// arrive, so the others run out of polls; no block waits without bound.
__device__ void grid_barrier(DevState* st, unsigned nblocks, long long spins_max, bool skip) {
  __syncthreads();
  if (nblocks > 1 && threadIdx.x == 0) {
    volatile unsigned* genp = &st->bar_gen;
    const unsigned gen = *genp;
    __threadfence();
    const unsigned arrived = skip ? 0u : atomicAdd(&st->bar_count, 1u);
    if (!skip && arrived == nblocks - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*genp == gen) {
        __nanosleep(32);
        if (++spins > spins_max) {
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

// One segment of a column: vertex ids, lambda numerators P + R z, and its z range [z0, z1].
template <int D>
struct Seg {
  int vid[D + 1];
  int P[D + 1];
  int R[D + 1];
  int z0, z1;
};

// Segments of the column with fixed offsets o[0..D-2] (the last axis, z, varies in [0,s)).
template <int D>
__device__ __forceinline__ int column_segments(const int* o, int s, Seg<D>* sg) {
  if constexpr (D == 2) {
    const int ox = o[0];
    // z <= ox: pi = (x, y)
    sg[0].vid[0] = 0; sg[0].vid[1] = 1; sg[0].vid[2] = 3;
    sg[0].P[0] = s - ox; sg[0].P[1] = ox; sg[0].P[2] = 0;
    sg[0].R[0] = 0; sg[0].R[1] = -1; sg[0].R[2] = 1;
    sg[0].z0 = 0; sg[0].z1 = ox;
    // z > ox: pi = (y, x)
    sg[1].vid[0] = 0; sg[1].vid[1] = 2; sg[1].vid[2] = 3;
    sg[1].P[0] = s; sg[1].P[1] = -ox; sg[1].P[2] = ox;
    sg[1].R[0] = -1; sg[1].R[1] = 1; sg[1].R[2] = 0;
    sg[1].z0 = ox + 1; sg[1].z1 = s - 1;
    return 2;
  } else {
    const int ox = o[0], oy = o[1];
    const bool xhi = ox >= oy;
    const int hi = xhi ? ox : oy, lo = xhi ? oy : ox;
    const int bh = xhi ? 1 : 2, bl = xhi ? 2 : 1;  // vertex bits of the hi / lo axis
    // A: z <= lo, pi = (hi, lo, z)
    sg[0].vid[0] = 0; sg[0].vid[1] = bh; sg[0].vid[2] = bh | bl; sg[0].vid[3] = 7;
    sg[0].P[0] = s - hi; sg[0].P[1] = hi - lo; sg[0].P[2] = lo; sg[0].P[3] = 0;
    sg[0].R[0] = 0; sg[0].R[1] = 0; sg[0].R[2] = -1; sg[0].R[3] = 1;
    sg[0].z0 = 0; sg[0].z1 = lo;
    // B: lo < z <= hi, pi = (hi, z, lo)
    sg[1].vid[0] = 0; sg[1].vid[1] = bh; sg[1].vid[2] = bh | 4; sg[1].vid[3] = 7;
    sg[1].P[0] = s - hi; sg[1].P[1] = hi; sg[1].P[2] = -lo; sg[1].P[3] = lo;
    sg[1].R[0] = 0; sg[1].R[1] = -1; sg[1].R[2] = 1; sg[1].R[3] = 0;
    sg[1].z0 = lo + 1; sg[1].z1 = hi;
    // C: z > hi, pi = (z, hi, lo)
    sg[2].vid[0] = 0; sg[2].vid[1] = 4; sg[2].vid[2] = 4 | bh; sg[2].vid[3] = 7;
    sg[2].P[0] = s; sg[2].P[1] = -hi; sg[2].P[2] = hi - lo; sg[2].P[3] = lo;
    sg[2].R[0] = -1; sg[2].R[1] = 1; sg[2].R[2] = 0; sg[2].R[3] = 0;
    sg[2].z0 = hi + 1; sg[2].z1 = s - 1;
    return 3;
  }
}

enum { kFirst = 0, kNewton = 1, kUpdate = 2 };

// (A_H c) at the interior coarse node z (offset off in the coarse nodal array c, boundary
// zero): sigma_H (2d c - sum of axis neighbours), or with the coefficient
// sigma_H sum_e w_e (c - c_e) (T_H is the coefficient's own mesh: level shift 0).
template <int D>
__device__ __forceinline__ double coarse_apply(const AugArgs& A, const double* c, long long off, const int* z) {
  const double sig = A.sigma_H;
  long long mul = 1;
  if (A.vc.a64) {
    double w[2 * D];
    edge_weights_t<D, double>(A.vc, 0, z[0], z[1], D == 3 ? z[2] : 0, w);
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < D; ++q) {
      acc += w[2 * q] * (c[off] - c[off - mul]) + w[2 * q + 1] * (c[off] - c[off + mul]);
      mul *= (A.nc + 1);
    }
    return sig * acc;
  }
  double nb = 0.0;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    nb += c[off - mul] + c[off + mul];
    mul *= (A.nc + 1);
  }
  return sig * (2.0 * D * c[off] - nb);
}

// Entry of A_H between the interior coarse node z and its box neighbour z + dv (|dv|_1 = dist):
// the diagonal, an axis neighbour's coupling, or zero (dist >= 2: the diagonal couplings of
// these meshes vanish for a diagonal coefficient).
template <int D>
__device__ __forceinline__ double coarse_stiffness(const AugArgs& A, const int* z, const int* dv, int dist) {
  const double sig = A.sigma_H;
  if (dist > 1) return 0.0;
  if (!A.vc.a64) return dist == 0 ? sig * 2.0 * D : -sig;
  double w[2 * D];
  edge_weights_t<D, double>(A.vc, 0, z[0], z[1], D == 3 ? z[2] : 0, w);
  if (dist == 1) {
    int e = 0;
#pragma unroll
    for (int q = 0; q < D; ++q)
      if (dv[q] != 0) e = 2 * q + (dv[q] > 0 ? 1 : 0);
    return -sig * w[e];
  }
  double sw = 0.0;
#pragma unroll
  for (int e = 0; e < 2 * D; ++e) sw += w[e];
  return sig * sw;
}

// Mixed path, passes after the first: the increment dF = a (f(u~ + d) - f(u~)) and a f'(u~ + d)
// in FP32, from closed forms that do not cancel (d is the small Newton correction
// (alpha - 1) u~ + P c).  The residual sums of the first pass (FP64, at U = u~) plus these
// increments give the residual at U to FP64-level accuracy.  signed |u|^{3/2} has no such
// form and is evaluated in FP64.
__device__ __forceinline__ void delta_f(int kind, double a, ff ut, float utf, float d, float af, float& dF,
                                        float& Fp) {
  switch (kind) {
    case FMG_F_CUBIC: {
      const float U = utf + d;
      dF = af * d * fmaf(3.0f * utf, U, d * d);
      Fp = 3.0f * af * U * U;
      break;
    }
    case FMG_F_EXPM1: {
      const float e = expf(utf);
      dF = af * e * expm1f(d);
      Fp = af * e * expf(d);
      break;
    }
    case FMG_F_LINEAR:
      dF = af * d;
      Fp = af;
      break;
    case FMG_F_NEG_EXP_NEG: {
      const float e = expf(-utf);
      dF = -af * e * expm1f(-d);
      Fp = af * e * expf(-d);
      break;
    }
    default: {  // FMG_F_SIGNED_POW32
      double F1, F0, Fp1, Fp0;
      const double u0 = ff_to_double(ut);
      f_eval<double>(kind, a, u0 + (double)d, F1, Fp1);
      f_eval<double>(kind, a, u0, F0, Fp0);
      dF = (float)(F1 - F0);
      Fp = (float)Fp1;
      break;
    }
  }
}

// Moments of the mixed first pass over a run of column nodes: the residual and t/s moments in
// float-float, the Jacobian moments in FP32.
struct FirstMoments {
  ff q0, q1, sa, t0, t1, ss;
  float d0, d1, d2, e0, e1, js;
};

// One node of the mixed first pass: u~ = U and g = G at the node, its axis neighbours um[ax]
// and up[ax], fine z coordinate z.  CUBIC selects a f(u) = a u^3 at compile time (no branch in
// the node's arithmetic); otherwise the nonlinearity is chosen by A.kind.  The Jacobian
// moments are formed also in the fixed-point iteration, which does not read them.
template <int D, bool CUBIC, bool VC>
__device__ __forceinline__ void first_node(const AugArgs& A, FirstMoments& m, ff U, ff G, const ff* um, const ff* up,
                                           int z, int x, int y, int zc) {
  ff F;
  float Fpf;
  if (CUBIC) {
    F = ff_mul(ff_mul(ff_mul(U, U), U), A.a_ff);
    Fpf = 3.0f * (A.a_ff.hi * (U.hi * U.hi));   // the FP32 derivative of the cubic, as f_eval forms it
  } else {
    F = f_ff(A.kind, A.a_ff, A.a, U);
    float Ff;
    f_eval<float>(A.kind, A.a_ff.hi, U.hi, Ff, Fpf);
  }
  // f(u~) - g enters the sums only: an add whose error is bounded relative to |f| + |g| (as
  // for an FP64 subtraction) suffices
  const ff Fm = ff_add_fast(F, ff_neg(G));
  const float zf = (float)z;
  m.q0 = ff_add_fast(m.q0, Fm);
  m.q1 = ff_add_fast(m.q1, ff_mul_f(Fm, zf));
  m.sa = ff_add_fast(m.sa, ff_mul(Fm, U));
  const float dz = Fpf * zf, du = Fpf * U.hi;
  m.d0 += Fpf;
  m.d1 += dz;
  m.d2 = fmaf(dz, zf, m.d2);
  m.e0 += du;
  m.e1 = fmaf(du, zf, m.e1);
  m.js = fmaf(du, U.hi, m.js);
  // A_k u~ = sigma (2d u - sum of axis neighbours) = -sigma * neighbour sum; with the
  // coefficient -sigma * sum_e w_e (u_e - u) at fine node (x, z) / (x, y, z) (z = zc + local z)
  ff nsum;
  if constexpr (VC) {
    ff nb[2 * D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      nb[2 * ax] = um[ax];
      nb[2 * ax + 1] = up[ax];
    }
    const int za = zc + z;
    nsum = weighted_neighbour_sum_ff<D>(U, nb, A.vc, A.ls, x, D == 2 ? za : y, D == 3 ? za : 0);
  } else {
    nsum = neighbour_sum_ff_v<D>(U, um, up);
  }
  if (D == 3) nsum = ff_mul(nsum, A.sigma_ff);
  const ff au = ff_neg(nsum);
  m.t0 = ff_add_fast(m.t0, au);
  m.t1 = ff_add_fast(m.t1, ff_mul_f(au, zf));
  m.ss = ff_add_fast(m.ss, ff_mul(au, U));
}

// A batch of up to B consecutive column nodes z .. z+cnt-1 (offset `off` at z) of the mixed
// first pass.  Every value the batch needs -- u~ at z-1 .. z+B, g and the in-plane axis
// neighbours at the B nodes -- is loaded into registers before the arithmetic, so the batch
// costs one memory latency; loads past the run (cnt < B) repeat its last valid node and their
// nodes are not summed.
template <int D, bool CUBIC, int B, bool VC>
__device__ __forceinline__ void first_batch(const AugArgs& A, FirstMoments& m, long long off, int z, int cnt,
                                            long long zstride, long long np, int x, int y, int zc) {
  constexpr int NI = D - 1;                  // in-plane axes: x (and y in 3D); the column is the last
  const long long io[2] = {1, np};
  ff uz[B + 2], gv[B], um[NI > 0 ? NI : 1][B], up[NI > 0 ? NI : 1][B];
#pragma unroll
  for (int q = 0; q < B + 2; ++q) uz[q] = ff_load(A.u + off + (long long)(min(q, cnt + 1) - 1) * zstride);
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const long long c = off + (long long)min(q, cnt - 1) * zstride;
    gv[q] = ff_load(A.g + c);
#pragma unroll
    for (int ax = 0; ax < NI; ++ax) {
      um[ax][q] = ff_load(A.u + c - io[ax]);
      up[ax][q] = ff_load(A.u + c + io[ax]);
    }
  }
#pragma unroll
  for (int q = 0; q < B; ++q) {
    if (q >= cnt) break;
    ff nm[D], nq[D];
#pragma unroll
    for (int ax = 0; ax < NI; ++ax) {
      nm[ax] = um[ax][q];
      nq[ax] = up[ax][q];
    }
    nm[D - 1] = uz[q];
    nq[D - 1] = uz[q + 2];
    first_node<D, CUBIC, VC>(A, m, uz[q + 1], gv[q], nm, nq, z + q, x, y, zc);
  }
}

// The mixed first pass over the column nodes z0..z1 (offset `off` at z0), in register batches
// of B nodes (B smaller in 3D, whose nodes have two more in-plane neighbours to hold).  x, y:
// the column's fine in-plane coordinates; zc: the fine z of local z = 0 (the coefficient's
// edge weights need the node's position).
template <int D, bool CUBIC, bool VC>
__device__ __forceinline__ void first_pass_segment(const AugArgs& A, long long off, int z0, int z1,
                                                   long long zstride, FirstMoments& m, int x, int y, int zc) {
  constexpr int B = D == 2 ? 8 : 4;
  const long long np = A.n + 1;
  m.q0 = m.q1 = m.sa = m.t0 = m.t1 = m.ss = ff{0.f, 0.f};
  m.d0 = m.d1 = m.d2 = m.e0 = m.e1 = m.js = 0.f;
  for (int z = z0; z <= z1; z += B, off += B * zstride)
    first_batch<D, CUBIC, B, VC>(A, m, off, z, min(B, z1 - z + 1), zstride, np, x, y, zc);
}

// The fine pass of one block: columns of its cell, chunk by chunk.  `acc` holds the
// per-thread channel rows ([NVAL][NT] doubles), zero on entry.
template <int D, bool JF32, bool VC = false>
__device__ void fine_pass(const AugArgs& A, int phase, double* acc, const double* cv, double alpha, int cell,
                          int bic) {
  using G = Aug<D, JF32>;
  using JT = typename std::conditional<JF32, float, double>::type;
  const int tid = threadIdx.x;
  const int s = A.s;
  const long long np = A.n + 1;
  const long long zstride = D == 2 ? np : np * np;
  int cellc[3] = {0, 0, 0};
  {
    int t = cell;
    for (int q = 0; q < D; ++q) {
      cellc[q] = t % A.nc;
      t /= A.nc;
    }
  }
  const int ncol = D == 2 ? s : s * s;
  const int nch = s / A.chunk;
  const long long items = (long long)ncol * nch;
  const double inv_s = 1.0 / s;
  const double inv_s2 = inv_s * inv_s;
  // the mixed path's FP32 quantities, formed once per pass: Jacobian weights, alpha - 1, a,
  // 1/s and the coarse cell's vertex values of c
  const float jw0 = JF32 ? (float)A.w : 0.f, jw1 = JF32 ? (float)(A.w * inv_s) : 0.f,
              jw2 = JF32 ? (float)(A.w * inv_s2) : 0.f;
  const float am1f = JF32 ? (float)(alpha - 1.0) : 0.f, a_f = JF32 ? (float)A.a : 0.f;
  const float inv_sf = 1.0f / (float)s;
  float cvf[G::NV];
#pragma unroll
  for (int v = 0; v < G::NV; ++v) cvf[v] = (JF32 && phase != kFirst) ? (float)cv[v] : 0.f;
  // Items (column chunks) are dealt to the cell's blocks contiguously when they fill every
  // block; on small levels they are interleaved across the blocks, so that the cell's work
  // spreads over as many SM sub-partitions as there are items (the FP64 rate of one
  // sub-partition is one warp instruction per 64 clocks, so a single busy warp per cell would
  // serialize the pass).
  const bool spread = items < (long long)A.bpc * G::NT;
  const long long q0 = spread ? (long long)tid * A.bpc + bic : (long long)bic * G::NT + tid;
  const long long qstep = (long long)A.bpc * G::NT;
  for (long long q = q0; q < items; q += qstep) {
    const int col = (int)(q % ncol);
    const int ch = (int)(q / ncol);
    const int o[2] = {col % s, D == 3 ? col / s : 0};
    // fine coordinates of the column; a column on the x = 0 (or y = 0) face is boundary
    const int x = cellc[0] * s + o[0];
    const int y = D == 3 ? cellc[1] * s + o[1] : 0;
    if (x == 0 || (D == 3 && y == 0)) continue;
    const int zc = cellc[D - 1] * s;                   // fine z of local offset 0
    const long long base = D == 2 ? (long long)x : (long long)y * np + x;
    const int zlo_chunk = ch * A.chunk;
    const int zhi_chunk = zlo_chunk + A.chunk - 1;
    const int zmin = (zc == 0) ? 1 : 0;                // z = 0 is the boundary face
    Seg<D> sg[D];
    const int nseg = column_segments<D>(o, s, sg);
    for (int si = 0; si < nseg; ++si) {
      const Seg<D>& S = sg[si];
      const int z0 = max(max(S.z0, zlo_chunk), zmin);
      const int z1 = min(S.z1, zhi_chunk);
      if (z0 > z1) continue;
      // P c on the segment: pc0 + pc1 z (the mixed path forms it in FP32: it is the small
      // Newton correction, and the passes after the first work in FP32 increments)
      double pc0 = 0.0, pc1 = 0.0;
      float pc0f = 0.f, pc1f = 0.f;
      if (JF32 && phase != kFirst) {
#pragma unroll
        for (int t = 0; t <= D; ++t) {
          pc0f = fmaf((float)S.P[t], cvf[S.vid[t]], pc0f);
          pc1f = fmaf((float)S.R[t], cvf[S.vid[t]], pc1f);
        }
        pc0f *= inv_sf;
        pc1f *= inv_sf;
      } else if (phase != kFirst) {
#pragma unroll
        for (int t = 0; t <= D; ++t) {
          pc0 += S.P[t] * cv[S.vid[t]];
          pc1 += S.R[t] * cv[S.vid[t]];
        }
        pc0 *= inv_s;
        pc1 *= inv_s;
      }
      double Q0 = 0.0, Q1 = 0.0, SAv = 0.0;                 // residual moments
      JT D0 = 0, D1 = 0, D2 = 0, E0 = 0, E1 = 0, JSv = 0;   // Jacobian moments
      double T0 = 0.0, T1 = 0.0, SSv = 0.0;                 // first pass
      FirstMoments fm;                                      // mixed path, first pass
      float cq0 = 0.f, cq1 = 0.f, csa = 0.f;                // mixed path, chord pass
      double zd = (double)z0;
      long long off = base + (long long)(zc + z0) * zstride;
      if (JF32 && phase != kFirst) {
        // mixed path: FP32 increments on top of the first pass's FP64 residual sums
        const float af = a_f;
        float q0 = 0.f, q1 = 0.f, sa = 0.f;
        auto node = [&](ff ut, float zf, long long o) {
          const float utf = ut.hi;
          const float dl = fmaf(am1f, utf, fmaf(pc1f, zf, pc0f));
          if (phase == kUpdate) {
            const ff un = ff_add_f(ut, dl);
            if (A.out_f64)
              A.u[o] = ff_to_double_fast(un);
            else
              ff_store(A.u + o, un);
            return;
          }
          // chord step: the Jacobian of the first pass is reused, so only the residual
          // increments are summed here
          float dF, fp;
          delta_f(A.kind, A.a, ut, utf, dl, af, dF, fp);
          q0 += dF;
          q1 = fmaf(dF, zf, q1);
          sa = fmaf(dF, utf, sa);
        };
        // sixteen independent loads in flight before the arithmetic, one memory latency per
        // batch; loads past the run repeat its last node and are not processed
        constexpr int BU = 16;
        for (int z = z0; z <= z1; z += BU, off += BU * zstride) {
          const int cnt = min(BU, z1 - z + 1);
          ff v[BU];
#pragma unroll
          for (int q = 0; q < BU; ++q) v[q] = ff_load(A.u + off + (long long)min(q, cnt - 1) * zstride);
#pragma unroll
          for (int q = 0; q < BU; ++q) {
            if (q >= cnt) break;
            node(v[q], (float)(z + q), off + q * zstride);
          }
        }
        cq0 = q0;
        cq1 = q1;
        csa = sa;
      } else if (JF32) {
        // mixed path, first pass: u~ and g are float-float, and f(u~) - g, A_k u~ and the
        // residual and t/s moments are formed in float-float (FP32 error-free transformations,
        // no FP64 arithmetic per node); the Jacobian moments in FP32 from the leading parts
        if (A.kind == FMG_F_CUBIC)
          first_pass_segment<D, true, VC>(A, off, z0, z1, zstride, fm, x, y, zc);
        else
          first_pass_segment<D, false, VC>(A, off, z0, z1, zstride, fm, x, y, zc);
        D0 = fm.d0;
        D1 = fm.d1;
        D2 = fm.d2;
        E0 = fm.e0;
        E1 = fm.e1;
        JSv = fm.js;
      } else
      for (int z = z0; z <= z1; ++z, off += zstride, zd += 1.0) {
        if (((z - z0) & 7) == 0) {
          // touch the next eight column entries (and their g values) so that their loads are
          // in flight together (they stay in L1 for the iterations below)
#pragma unroll
          for (int q = 1; q < 8; ++q)
            if (z + q <= z1) {
              asm volatile("prefetch.global.L1 [%0];" ::"l"(A.u + off + q * zstride));
              if (phase != kUpdate) asm volatile("prefetch.global.L1 [%0];" ::"l"(A.g + off + q * zstride));
            }
        }
        const double ut = A.u[off];
        const double U = phase == kFirst ? ut : fma(alpha, ut, fma(pc1, zd, pc0));
        if (phase == kUpdate) {
          A.u[off] = U;
          continue;
        }
        // FP64 path (the mixed path's passes are the branches above)
        double F, Fp = 0.0;
        f_eval<double>(A.kind, A.a, U, F, Fp);
        const JT dj = (JT)Fp, zj = (JT)zd, uj = (JT)ut;
        const double Fm = F - A.g[off];
        Q0 += Fm;
        Q1 = fma(Fm, zd, Q1);
        SAv = fma(Fm, ut, SAv);
        if (!A.fixed_point) {
          const JT dz = dj * zj;
          const JT du = dj * uj;
          D0 += dj;
          D1 += dz;
          D2 += dz * zj;
          E0 += du;
          E1 += du * zj;
          JSv += du * uj;
        }
        if (phase == kFirst) {
          double au;
          if constexpr (VC) {
            // sigma sum_e w_e (u - u_e) with the coefficient's edge weights at the node
            double wt[2 * D];
            const int za = zc + z;
            edge_weights_t<D, double>(A.vc, A.ls, x, D == 2 ? za : y, D == 3 ? za : 0, wt);
            const long long o3[3] = {1, np, zstride};
            double acc2 = 0.0;
#pragma unroll
            for (int ax = 0; ax < D; ++ax)
              acc2 += wt[2 * ax] * (ut - A.u[off - o3[ax]]) + wt[2 * ax + 1] * (ut - A.u[off + o3[ax]]);
            au = A.sigma_k * acc2;
          } else {
            double nb;
            if constexpr (D == 2) {
              nb = (A.u[off - 1] + A.u[off + 1]) + (A.u[off - zstride] + A.u[off + zstride]);
            } else {
              nb = ((A.u[off - 1] + A.u[off + 1]) + (A.u[off - np] + A.u[off + np])) +
                   (A.u[off - zstride] + A.u[off + zstride]);
            }
            au = A.sigma_k * (2.0 * D * ut - nb);
          }
          T0 += au;
          T1 = fma(au, zd, T1);
          SSv = fma(au, ut, SSv);
        }
      }
      if (phase == kUpdate) continue;
      // moments -> vertex channels of this thread's row
      const double w = A.w;
      if (JF32) {
        // mixed path: the residual (and first-pass t, s) channels are float-float rows without
        // their weights; the chord pass's moments are FP32 sums of increments
        float2* fr = reinterpret_cast<float2*>(acc);
        auto add = [&](int ch, ff x) {
          const float2 o = fr[ch * G::NT + tid];
          const ff r = ff_add_fast(ff{o.x, o.y}, x);
          fr[ch * G::NT + tid] = make_float2(r.hi, r.lo);
        };
        if (phase != kFirst) {
#pragma unroll
          for (int t = 0; t <= D; ++t)
            add(G::RA + S.vid[t], ff{fmaf((float)S.P[t], cq0, (float)S.R[t] * cq1), 0.f});
          add(G::SA, ff{csa, 0.f});
          continue;
        }
#pragma unroll
        for (int t = 0; t <= D; ++t) {
          const float Pt = (float)S.P[t], Rt = (float)S.R[t];
          const int v = S.vid[t];
          add(G::RA + v, ff_add(ff_mul_f(fm.q0, Pt), ff_mul_f(fm.q1, Rt)));
          add(G::TT + v, ff_add(ff_mul_f(fm.t0, Pt), ff_mul_f(fm.t1, Rt)));
        }
        add(G::SA, fm.sa);
        add(G::SS, fm.ss);
      } else {
#pragma unroll
        for (int t = 0; t <= D; ++t) {
          const double Pt = S.P[t], Rt = S.R[t];
          const int v = S.vid[t];
          acc[(G::RA + v) * G::NT + tid] += w * inv_s * (Pt * Q0 + Rt * Q1);
          if (phase == kFirst) acc[(G::TT + v) * G::NT + tid] += inv_s * (Pt * T0 + Rt * T1);
        }
        acc[G::SA * G::NT + tid] += w * SAv;
        if (phase == kFirst) acc[G::SS * G::NT + tid] += SSv;
      }
      if (A.fixed_point) continue;   // the fixed-point iteration needs no Jacobian
      if (JF32) {
        // FP32 Jacobian channels, converted in FP32 into the FP32 rows
        float* fj = Rows<D, JF32>::jac(acc);
        const float wf = jw1, wf2 = jw2;
        const float d0 = (float)D0, d1 = (float)D1, d2 = (float)D2, e0 = (float)E0, e1 = (float)E1;
#pragma unroll
        for (int t = 0; t <= D; ++t) {
          const float Pt = (float)S.P[t], Rt = (float)S.R[t];
          const int v = S.vid[t];
          fj[(G::JB - G::JB + v) * G::NT + tid] += wf * fmaf(Pt, e0, Rt * e1);
#pragma unroll
          for (int r = t; r <= D; ++r) {
            const float Pr = (float)S.P[r], Rr = (float)S.R[r];
            fj[(G::JP - G::JB + pair_index(G::NV, v, S.vid[r])) * G::NT + tid] +=
                wf2 * fmaf(Pt * Pr, d0, fmaf(fmaf(Pt, Rr, Rt * Pr), d1, Rt * Rr * d2));
          }
        }
        fj[(G::JS - G::JB) * G::NT + tid] += jw0 * (float)JSv;
      } else {
#pragma unroll
        for (int t = 0; t <= D; ++t) {
          const double Pt = S.P[t], Rt = S.R[t];
          const int v = S.vid[t];
          acc[(G::JB + v) * G::NT + tid] += w * inv_s * (Pt * (double)E0 + Rt * (double)E1);
#pragma unroll
          for (int r = t; r <= D; ++r) {
            const double Pr = S.P[r], Rr = S.R[r];
            acc[(G::JP + pair_index(G::NV, v, S.vid[r])) * G::NT + tid] +=
                w * inv_s2 * (Pt * Pr * (double)D0 + (Pt * Rr + Rt * Pr) * (double)D1 + Rt * Rr * (double)D2);
          }
        }
        acc[G::JS * G::NT + tid] += w * (double)JSv;
      }
    }
  }
}

// Block sum of the channel rows into out[0..NVAL) (fixed order).  Only the channels the
// phase produced are summed (the first-pass gatherings t and s only in the first
// pass); in the mixed path the Jacobian channels, FP32 products to begin with, are summed in
// FP32 -- FP64 adds issue slowly on this part.
template <int D, bool JF32>
__device__ void block_reduce_rows(const AugArgs& A, const double* acc, double* out, bool first, bool fixed_point) {
  using G = Aug<D, JF32>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = G::NT / 32;
  __syncthreads();
  for (int v = warp; v < G::NVAL; v += nw) {
    const bool pre = v >= G::TT && v < G::JB;
    if (pre && !first) continue;
    if ((fixed_point || (JF32 && !first)) && v >= G::JB) continue;   // no Jacobian channels
    if (JF32 && v >= G::JB) {
      const float* fj = Rows<D, JF32>::jac(acc);
      float x = 0.f;
      for (int t = lane; t < G::NT; t += 32) x += fj[(v - G::JB) * G::NT + t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      // the FP32 sum stays FP32: it is stored in the low word of the channel's 8-byte slot
      if (lane == 0) reinterpret_cast<float*>(out + v)[0] = x;
    } else if (JF32) {
      // float-float rows: summed in float-float (fixed order), then weighted and converted
      const float2* fr = reinterpret_cast<const float2*>(acc);
      ff x{0.f, 0.f};
      for (int t = lane; t < G::NT; t += 32) {
        const float2 o = fr[v * G::NT + t];
        x = ff_add_fast(x, ff{o.x, o.y});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const ff y{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
        x = ff_add_fast(x, y);
      }
      if (lane == 0) {
        const double inv_s = 1.0 / A.s;
        const double wgt = v < G::SA ? A.w * inv_s : v == G::SA ? A.w : v < G::SS ? inv_s : 1.0;
        out[v] = wgt * ff_to_double(x);
      }
    } else {
      double x = 0.0;
      for (int t = lane; t < G::NT; t += 32) x += acc[v * G::NT + t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) out[v] = x;
    }
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

template <int D>
__device__ __forceinline__ long long coarse_offset(const int* z, int nc) {
  const long long cp = nc + 1;
  long long off = 0, mul = 1;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    off += (long long)z[q] * mul;
    mul *= cp;
  }
  return off;
}

// Sum of channel `ch` at vertex p over the cells around coarse node p.
template <int D, bool JF32>
__device__ double node_channel(const double* cellsum, int nc, const int* z, int ch) {
  using G = Aug<D, JF32>;
  double x = 0.0;
  for (int o = 0; o < G::NV; ++o) {
    bool ok = true;
    int cell = 0, mul = 1;
    for (int q = 0; q < D; ++q) {
      const int cc = z[q] - ((o >> q) & 1);
      if (cc < 0 || cc >= nc) ok = false;
      cell += cc * mul;
      mul *= nc;
    }
    if (ok) x += cellsum[(long long)cell * G::NVAL + ch + o];
  }
  return x;
}

template <int D, bool JF32>
__device__ double pair_channel(const double* cellsum, int nc, const int* zp, const int* zq) {
  using G = Aug<D, JF32>;
  double x = 0.0;
  for (int o = 0; o < G::NV; ++o) {
    bool ok = true;
    int cell = 0, mul = 1, vq = 0;
    for (int q = 0; q < D; ++q) {
      const int cc = zp[q] - ((o >> q) & 1);
      if (cc < 0 || cc >= nc) ok = false;
      const int dq = zq[q] - cc;
      if (dq < 0 || dq > 1) ok = false;
      vq |= dq << q;
      cell += cc * mul;
      mul *= nc;
    }
    if (ok) x += cellsum[(long long)cell * G::NVAL + G::JP + pair_index(G::NV, o, vq)];
  }
  return x;
}

// Lexicographic half-bandwidth of J_HH: it couples coarse nodes that share a coarse simplex,
// offsets up to 1 + m (2D) or 1 + m + m^2 (3D), m = nc - 1; alpha is the border unknown.
template <int D>
__device__ __forceinline__ int aug_band(int nc) {
  const int m = nc - 1;
  return D == 2 ? m + 1 : m * m + m + 1;
}

// Block-local state of the Newton iteration, in shared memory past the channel rows, kept
// from pass to pass.  Every block of the grid (every CTA of a cluster) takes the same Newton
// step from the same partial sums in the same order, so all hold the same iterate and reach
// the same decisions: no second barrier and no global copy of the iterate are needed.
struct StepState {
  double* c;       // coarse nodal iterate ((nc+1)^d values, boundary 0)
  double* t;       // t = P^T A_k u~  [N_H]
  double* sa;      // [0] s = u~.A_k u~, [1] alpha
  double* basev;   // mixed path: the first pass's FP64 residual sums [ncell (NV+1)]
  int* flags;      // [0] converged, [1] stop (a pivot was not positive or a value not finite)
};

// Shared memory of the Newton kernels: the channel rows (reused after each pass for cellsum
// [ncell NVAL], M [NA (NA+1)] and R [NA+1]), then the StepState arrays, then the factor L
// [NA (NA+1)] and its reciprocal pivots [NA] in the factor's precision.
template <int D, bool JF32>
struct AugSmem {
  using G = Aug<D, JF32>;
  using FT = typename std::conditional<JF32, float, double>::type;
  __host__ __device__ static int ncell(int nc) { return (int)ipow(nc, D); }
  __host__ __device__ static int NA(int nc) { return (int)ipow(nc - 1, D) + 1; }
  __host__ __device__ static size_t region(int nc) {
    const size_t na = (size_t)NA(nc);
    const size_t scratch = sizeof(double) * ((size_t)ncell(nc) * G::NVAL + na * (na + 1) + na + 1);
    const size_t r = Rows<D, JF32>::bytes > scratch ? Rows<D, JF32>::bytes : scratch;
    return (r + 15) & ~size_t(15);
  }
  __host__ __device__ static size_t state_doubles(int nc) {
    return (size_t)ipow(nc + 1, D) + (size_t)(NA(nc) - 1) + 2 + (size_t)ncell(nc) * (G::NV + 1);
  }
  __host__ __device__ static size_t bytes(int nc) {
    const size_t na = (size_t)NA(nc);
    return region(nc) + sizeof(double) * state_doubles(nc) + sizeof(FT) * (na * (na + 1) + na);
  }
  __device__ static void carve(double* sm, int nc, StepState& S, FT*& L) {
    char* base = reinterpret_cast<char*>(sm) + region(nc);
    S.c = reinterpret_cast<double*>(base);
    S.t = S.c + ipow(nc + 1, D);
    S.sa = S.t + (NA(nc) - 1);
    S.basev = S.sa + 2;
    L = reinterpret_cast<FT*>(S.basev + (size_t)ncell(nc) * (G::NV + 1));
  }
};

// Sum over the bpc blocks of a cell of one channel of their partial rows, in block order, with
// the loads of four blocks issued together.  FP32: the channel's FP32 value in the low word of
// each slot.
template <int NVAL, bool F32>
__device__ __forceinline__ double sum_blocks(const double* __restrict__ p, int bpc) {
  double x = 0.0;
  float xf = 0.f;
  int b = 0;
  auto add = [&](double v) {
    if (F32)
      xf += __int_as_float(__double2loint(v));
    else
      x += v;
  };
  for (; b + 4 <= bpc; b += 4) {
    const double v0 = __ldcg(p + (size_t)(b + 0) * NVAL), v1 = __ldcg(p + (size_t)(b + 1) * NVAL);
    const double v2 = __ldcg(p + (size_t)(b + 2) * NVAL), v3 = __ldcg(p + (size_t)(b + 3) * NVAL);
    add(v0);
    add(v1);
    add(v2);
    add(v3);
  }
  for (; b < bpc; ++b) add(__ldcg(p + (size_t)b * NVAL));
  return F32 ? __hiloint2double(0, __float_as_int(xf)) : x;
}

// Several blocks per coarse cell: after its block sum, each block arrives at its cell's counter,
// and the one that arrives last sums the cell's partial rows (block order, the channels this
// pass filled) into the cell's row of cbuf and resets the counter, all before the grid barrier.
// After the barrier every block reads one row per cell instead of the rows of every block.
template <int D, bool JF32>
__device__ void cell_reduce(const AugArgs& A, const double* __restrict__ pbuf, double* __restrict__ cbuf, int cell,
                            bool first, int* last_sh) {
  using G = Aug<D, JF32>;
  __threadfence();   // this block's partial row before its arrival
  __syncthreads();
  if (threadIdx.x == 0) *last_sh = atomicAdd(&A.st->cell_count[cell], 1u) == (unsigned)(A.bpc - 1) ? 1 : 0;
  __syncthreads();
  if (!*last_sh) return;
  __threadfence();   // the other blocks' rows, after their arrivals
  const bool fixed_point = A.fixed_point != 0;
  const double* rows = pbuf + (size_t)cell * A.bpc * G::NVAL;
  for (int v = threadIdx.x; v < G::NVAL; v += blockDim.x) {
    if (v >= G::TT && v < G::JB && !first) continue;                   // t, s: first pass only
    if (v >= G::JB && (fixed_point || (JF32 && !first))) continue;      // no Jacobian channels
    cbuf[(size_t)cell * G::NVAL + v] = (JF32 && v >= G::JB) ? sum_blocks<G::NVAL, true>(rows + v, A.bpc)
                                                            : sum_blocks<G::NVAL, false>(rows + v, A.bpc);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicExch(&A.st->cell_count[cell], 0u);
}

template <int D>
__device__ void newton_update(const AugArgs& A, const double* R, int NH, const StepState& S, int dropped, bool ok,
                              bool writer);

// Gather table of the mixed path's FP32 Jacobian (first iteration of a correction step): one
// record of kJW<D> ints per entry e of the assembly, e = p (3^d + 1) + r for coarse unknown p and
// r < 3^d its neighbour z_p + (r digits in base 3) - 1, r = 3^d the border entry of p:
//   [0] the entry's index into the factor's array (p ld + q, or N_H ld + p), -1: outside the
//       lower band or the mesh;
//   [1] |dv|_1 (bits 0-1), border flag (bit 2), p (bits 8-15), r (bits 16-23);
//   [2 + o] for each of the 2^d cells around the node (o: the vertex bits of p in the cell), the
//       cell-sum slot of the channel the entry takes from that cell, or -1.
// The entry is the sum of those FP32 channels in o order (the same order as summing cell by
// cell), so a table-driven assembly does no index arithmetic on the coarse mesh.
template <int D>
constexpr int kJW = D == 2 ? 8 : 12;

template <int D>
__host__ __device__ constexpr int aug_jtab_entries(int nc) {
  int nh = 1, n3 = 1;
  for (int q = 0; q < D; ++q) {
    nh *= nc - 1;
    n3 *= 3;
  }
  return nh * (n3 + 1);
}

template <int D>
__global__ void k_aug_jtab(int nc, int* __restrict__ tab) {
  pdl_start();
  using G = Aug<D, true>;
  constexpr int N3 = D == 2 ? 9 : 27;
  const int NH = (int)ipow(nc - 1, D);
  const int ld = NH + 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NH * (N3 + 1); e += gridDim.x * blockDim.x) {
    int* w = tab + (size_t)e * kJW<D>;
    for (int i = 0; i < kJW<D>; ++i) w[i] = -1;
    const int p = e / (N3 + 1), rr = e - p * (N3 + 1);
    int z[3];
    unknown_coords<D>(p, nc, z);
    if (rr == N3) {   // border entry: the channel JB of the vertex z in each cell around it
      w[0] = NH * ld + p;
      w[1] = 4 | (p << 8) | (rr << 16);
      for (int o = 0; o < G::NV; ++o) {
        bool ok = true;
        int cell = 0, mul = 1;
        for (int q = 0; q < D; ++q) {
          const int cc = z[q] - ((o >> q) & 1);
          if (cc < 0 || cc >= nc) ok = false;
          cell += cc * mul;
          mul *= nc;
        }
        if (ok) w[2 + o] = cell * G::NVAL + G::JB + o;
      }
      continue;
    }
    int zq[3], q = 0, mulq = 1, dist = 0, r2 = rr;
    bool okq = true;
    for (int ax = 0; ax < D; ++ax) {
      const int d = r2 % 3 - 1;
      r2 /= 3;
      zq[ax] = z[ax] + d;
      if (zq[ax] < 1 || zq[ax] > nc - 1) okq = false;
      q += (zq[ax] - 1) * mulq;
      mulq *= (nc - 1);
      dist += d < 0 ? -d : d;
    }
    if (!okq || q > p) continue;
    w[0] = p * ld + q;
    w[1] = (dist > 2 ? 2 : dist) | (p << 8) | (rr << 16);
    // the pair channel of (z, zq) in each cell that holds both
    for (int o = 0; o < G::NV; ++o) {
      bool ok = true;
      int cell = 0, mul = 1, vq = 0;
      for (int qq = 0; qq < D; ++qq) {
        const int cc = z[qq] - ((o >> qq) & 1);
        if (cc < 0 || cc >= nc) ok = false;
        const int dq = zq[qq] - cc;
        if (dq < 0 || dq > 1) ok = false;
        vq |= dq << qq;
        cell += cc * mul;
        mul *= nc;
      }
      if (ok) w[2 + o] = cell * G::NVAL + G::JP + pair_index(G::NV, o, vq);
    }
  }
}

// Largest lexicographic half-bandwidth of J_HH (aug_band) of a dimension: 2D 1/H <= 8 gives
// 8, 3D 1/H <= 4 gives 13.
template <int D>
__host__ __device__ constexpr int aug_band_max() {
  return D == 2 ? 8 : 13;
}

// Column c of J^{-1} from the band LDL^T factor of ldlt_band_warp (A in place: A[i][k] =
// L_ik d_k below the diagonal, rd[k] = 1/d_k; band rows 0..nb-1, dense border row nb = n - 1):
// the forward substitution L w = e_c with y = D^{-1} w kept in X's column, then the backward
// substitution L^T x = y over the band and the border entry.  The band window of the last KB
// values is kept in registers; every thread walks the same rows, so the factor's entries are
// shared-memory broadcasts.
template <int D>
__device__ __forceinline__ void band_inverse_column(const float* __restrict__ Af, const float* __restrict__ rd, int n,
                                                    int ld, int band, int c, float* __restrict__ X) {
  constexpr int KB = aug_band_max<D>();
  const int nb = n - 1;
  // win[t] holds the value of the row t + 1 steps back (forward) or ahead (backward); the
  // newest one (t = 0) enters each sum last, so the rest of the sum does not wait for it
  float win[KB];
#pragma unroll
  for (int t = 0; t < KB; ++t) win[t] = 0.f;
  for (int k = 0; k < nb; ++k) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int t = KB - 1; t >= 1; --t) {
      const int j = k - 1 - t;
      if (t < band && j >= 0) {
        if (t & 1)
          s1 = fmaf(Af[k * ld + j], win[t], s1);
        else
          s0 = fmaf(Af[k * ld + j], win[t], s0);
      }
    }
    const float a0 = k >= 1 ? Af[k * ld + k - 1] : 0.f;
    const float y = ((k == c ? 1.f : 0.f) - fmaf(a0, win[0], s0 + s1)) * rd[k];
    X[k * ld + c] = y;
#pragma unroll
    for (int t = KB - 1; t > 0; --t) win[t] = win[t - 1];
    win[0] = y;
  }
  {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int j = 0;
    for (; j + 3 < nb; j += 4) {
      s0 = fmaf(Af[nb * ld + j], X[j * ld + c], s0);
      s1 = fmaf(Af[nb * ld + j + 1], X[(j + 1) * ld + c], s1);
      s2 = fmaf(Af[nb * ld + j + 2], X[(j + 2) * ld + c], s2);
      s3 = fmaf(Af[nb * ld + j + 3], X[(j + 3) * ld + c], s3);
    }
    for (; j < nb; ++j) s0 = fmaf(Af[nb * ld + j], X[j * ld + c], s0);
    X[nb * ld + c] = ((nb == c ? 1.f : 0.f) - ((s0 + s1) + (s2 + s3))) * rd[nb];
  }
  const float xb = X[nb * ld + c];
#pragma unroll
  for (int t = 0; t < KB; ++t) win[t] = 0.f;
  for (int k = nb - 1; k >= 0; --k) {
    float s0 = Af[nb * ld + k] * xb, s1 = 0.f;
#pragma unroll
    for (int t = KB - 1; t >= 1; --t) {
      const int i = k + 1 + t;
      if (t < band && i < nb) {
        if (t & 1)
          s1 = fmaf(Af[i * ld + k], win[t], s1);
        else
          s0 = fmaf(Af[i * ld + k], win[t], s0);
      }
    }
    const float a0 = k + 1 < nb ? Af[(k + 1) * ld + k] : 0.f;
    const float x = X[k * ld + c] - rd[k] * fmaf(a0, win[0], s0 + s1);
    X[k * ld + c] = x;
#pragma unroll
    for (int t = KB - 1; t > 0; --t) win[t] = win[t - 1];
    win[0] = x;
  }
}

// The same column for a size and band fixed at compile time (the dense systems of the
// benchmark shapes).  The band window lives in W = BAND + 1 registers addressed modulo W, and
// the substitutions are unrolled W steps at a time, so every window slot and every offset into
// the factor is a compile-time constant: the loads of a step are issued ahead and only the FMA
// chain through the newest value stays on the critical path.
template <int NA, int BAND>
__device__ __forceinline__ void band_inverse_column_fixed(const float* __restrict__ Af, const float* __restrict__ rd,
                                                          int c, float* __restrict__ X) {
  constexpr int ld = NA + 1, nb = NA - 1, W = BAND + 1;
  float win[W];
#pragma unroll
  for (int m = 0; m < W; ++m) win[m] = 0.f;
  // one forward step: y_k = ([k == c] - sum_{t=1..BAND} A[k][k-t] y_{k-t}) / d_k; the older
  // terms go into two partial sums, the newest (t = 1) is added last; `guard`: rows near the top,
  // where k - t < 0 (decided at compile time in the peeled first block)
  auto fwd = [&](int k, int kk, bool guard) {
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int t = BAND; t >= 2; --t) {
      if (guard && k - t < 0) continue;
      if (t & 1)
        p1 = fmaf(Af[k * ld + k - t], win[(kk - t + W) % W], p1);
      else
        p0 = fmaf(Af[k * ld + k - t], win[(kk - t + W) % W], p0);
    }
    float sum = p0 + p1;
    if (!guard || k >= 1) sum = fmaf(Af[k * ld + k - 1], win[(kk - 1 + W) % W], sum);
    const float y = ((k == c ? 1.f : 0.f) - sum) * rd[k];
    win[kk] = y;
    X[k * ld + c] = y;
  };
#pragma unroll
  for (int kk = 0; kk < W; ++kk)
    if (kk < nb) fwd(kk, kk, true);
  for (int k0 = W; k0 < nb; k0 += W) {
#pragma unroll
    for (int kk = 0; kk < W; ++kk)
      if (k0 + kk < nb) fwd(k0 + kk, kk, false);
  }
  {
    float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int j = 0; j < nb; ++j) s4[j & 3] = fmaf(Af[nb * ld + j], X[j * ld + c], s4[j & 3]);
    X[nb * ld + c] = ((nb == c ? 1.f : 0.f) - ((s4[0] + s4[1]) + (s4[2] + s4[3]))) * rd[nb];
  }
  const float xb = X[nb * ld + c];
  // one backward step: x_k = y_k - (sum_{t=1..BAND} A[k+t][k] x_{k+t} + A[nb][k] x_nb) / d_k,
  // from the top (guard: rows where k + t >= nb)
#pragma unroll
  for (int m = 0; m < W; ++m) win[m] = 0.f;
  auto bwd = [&](int k, int kk, bool guard) {
    float p0 = Af[nb * ld + k] * xb, p1 = 0.f;
#pragma unroll
    for (int t = BAND; t >= 2; --t) {
      if (guard && k + t >= nb) continue;
      if (t & 1)
        p1 = fmaf(Af[(k + t) * ld + k], win[(kk - t + W) % W], p1);
      else
        p0 = fmaf(Af[(k + t) * ld + k], win[(kk - t + W) % W], p0);
    }
    float sum = p0 + p1;
    if (!guard || k + 1 < nb) sum = fmaf(Af[(k + 1) * ld + k], win[(kk - 1 + W) % W], sum);
    const float x = X[k * ld + c] - rd[k] * sum;
    win[kk] = x;
    X[k * ld + c] = x;
  };
#pragma unroll
  for (int kk = 0; kk < W; ++kk)
    if (nb - 1 - kk >= 0) bwd(nb - 1 - kk, kk, true);
  for (int k0 = nb - 1 - W; k0 >= 0; k0 -= W) {
#pragma unroll
    for (int kk = 0; kk < W; ++kk)
      if (k0 - kk >= 0) bwd(k0 - kk, kk, false);
  }
}

// Column c of J^{-1}: the unrolled form for the sizes it is instantiated for, else the loop.
template <int D>
__device__ __forceinline__ void band_inverse_dispatch(const float* Af, const float* rd, int n, int ld, int band, int c,
                                                      float* X) {
  if constexpr (D == 2) {
    if (n == 50 && band == 8) return band_inverse_column_fixed<50, 8>(Af, rd, c, X);
    if (n == 10 && band == 4) return band_inverse_column_fixed<10, 4>(Af, rd, c, X);
  } else {
    if (n == 28 && band == 13) return band_inverse_column_fixed<28, 13>(Af, rd, c, X);
  }
  band_inverse_column<D>(Af, rd, n, ld, band, c, X);
}

// y = X r for the n x n matrix X (leading dimension ld) and r in FP32, by all warps (a row per
// warp, the columns over its lanes, a shuffle sum in fixed order).
__device__ __forceinline__ void small_matvec(const float* X, int n, int ld, const float* r, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < n; i += nw) {
    float y = 0.f;
    if (lane < n) y = X[i * ld + lane] * r[lane];
    if (lane + 32 < n) y = fmaf(X[i * ld + lane + 32], r[lane + 32], y);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (lane == 0) out[i] = y;
  }
}

// (c, alpha) += y (FP64) and the convergence test ||y||_inf <= tol max(1, ||(c, alpha)||_inf),
// every thread taking unknowns; the maxima of the nonnegative FP32 magnitudes are formed with
// integer atomics on their bit patterns (order-independent).  red: three words, zero on entry.
template <int D>
__device__ void newton_update_mixed(const AugArgs& A, const float* y, int NH, const StepState& S, int dropped,
                                    bool ok, bool writer, unsigned* red) {
  const int tid = threadIdx.x;
  for (int p = tid; p <= NH; p += blockDim.x) {
    double nv;
    if (p < NH) {
      int z[3];
      unknown_coords<D>(p, A.nc, z);
      const long long off = coarse_offset<D>(z, A.nc);
      nv = S.c[off] + (double)y[p];
      S.c[off] = nv;
    } else {
      nv = S.sa[1] + (double)y[NH];
      S.sa[1] = nv;
    }
    const float dv = fabsf(y[p]), av = fabsf((float)nv);
    if (!(dv <= 3.0e38f) || !(av <= 3.0e38f)) atomicOr(&red[2], 1u);
    atomicMax(&red[0], __float_as_uint(dv));
    atomicMax(&red[1], __float_as_uint(av));
  }
  __syncthreads();
  if (tid == 0) {
    const bool finite = red[2] == 0u;
    const float dmax = __uint_as_float(red[0]), ymax = __uint_as_float(red[1]);
    S.flags[1] = (!ok || !finite) ? 1 : 0;
    S.flags[0] = (finite && dmax <= (float)A.tol * fmaxf(1.f, ymax)) ? 1 : 0;
    if (writer) {
      if (dropped) atomicOr(&A.st->flags, kFlagDropped);
      if (!ok) atomicOr(&A.st->flags, kFlagNotSPD);
      if (!finite) atomicOr(&A.st->flags, kFlagNonfinite);
    }
  }
}

// The dense step of the mixed path, after a pass, in every block.  The residual R of the
// (N_H+1)-dimensional system of eq. 3.6 on V_H + span{u~} is formed in FP64 from the cell
// sums (the first pass's sums are kept and the later passes' increments added to them).  The
// first iteration also assembles the Jacobian (fixed point: the Galerkin stiffness) in FP32
// from the FP32 channels directly into the band-plus-border pattern, factors it by the band
// LDL^T on one warp and forms its inverse from the factor (a column per thread), which is
// kept in shared memory: every iteration's step is then y = J^{-1} R, a block-wide
// matrix-vector product, so the later iterations are chord steps at the cost of one product.
// If the last pivot (the Schur complement of alpha) falls below 1e-6 of its original
// diagonal entry, alpha is frozen (its row and column of the inverse are zero).
template <int D>
__device__ __noinline__ void newton_step_mixed(const AugArgs& A, const double* __restrict__ partials,
                                               double* cellsum, double* Mreg, double* R, float* L,
                                               const StepState& S, bool first, bool writer) {
  using G = Aug<D, true>;
  constexpr int N3 = D == 2 ? 9 : 27;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int lane = tid & 31;
  const int ncell = (int)ipow(A.nc, D);
  const int NH = (int)ipow(A.nc - 1, D);
  const int NA = NH + 1;
  const int ld = NA + 1;
  const bool fixedp = A.fixed_point != 0;
  float* X = reinterpret_cast<float*>(Mreg);   // J^{-1} as it is formed [NA][ld]
  float* rf = X + (size_t)NA * ld;             // R in FP32 [NA]
  float* dl = rf + NA;                         // the step y = J^{-1} R [NA]
  __shared__ float s3_sh;
  __shared__ int fac_sh[2];
  __shared__ unsigned red_sh[3];
  if (tid == 0) red_sh[0] = red_sh[1] = red_sh[2] = 0u;
  // ---- cell sums (one row per coarse cell): the residual channels in FP64, in the first
  // iteration also t, s (FP64) and the Jacobian channels (FP32, low word of the slot); eight
  // items per thread are loaded together and copied as they are.
  const int nneed = first ? G::NVAL : G::NV + 1;
  const int total = ncell * nneed;
  for (int base = tid; base < total; base += 8 * nthr) {
    int dst[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int idx = base + r * nthr;
      dst[r] = -1;
      if (idx < total) {
        const int cell = idx / nneed, q = idx - cell * nneed;
        const int v = first ? q : (q < G::NV ? G::RA + q : G::SA);
        if (!(fixedp && v >= G::JB)) dst[r] = cell * G::NVAL + v;
      }
    }
    unsigned long long wv[8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
      wv[r] = dst[r] >= 0 ? __ldcg(reinterpret_cast<const unsigned long long*>(partials) + dst[r]) : 0ull;
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (dst[r] >= 0) reinterpret_cast<unsigned long long*>(cellsum)[dst[r]] = wv[r];
  }
  __syncthreads();
  // the first pass's residual sums are kept in basev; the later passes' increments are added
  // to them (fixed order, same thread each time)
  for (int idx = tid; idx < ncell * (G::NV + 1); idx += nthr) {
    const int cell = idx / (G::NV + 1), v = idx % (G::NV + 1);
    const long long ch = (long long)cell * G::NVAL + (v < G::NV ? G::RA + v : G::SA);
    if (first)
      S.basev[idx] = cellsum[ch];
    else
      cellsum[ch] += S.basev[idx];
  }
  if (first) {
    for (int p = tid; p < NH; p += nthr) {
      int z[3];
      unknown_coords<D>(p, A.nc, z);
      S.t[p] = node_channel<D, true>(cellsum, A.nc, z, G::TT);
    }
    if (tid >= nthr - 32) {
      double s0 = 0.0;
      float s3 = 0.f;
      for (int c = lane; c < ncell; c += 32) {
        s0 += cellsum[(long long)c * G::NVAL + G::SS];
        if (!fixedp) s3 += reinterpret_cast<const float*>(cellsum + (long long)c * G::NVAL + G::JS)[0];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      }
      if (lane == 0) {
        S.sa[0] = s0;
        s3_sh = s3;
      }
    }
    // the factor's pattern: everything outside it reads as zero
    for (int i = tid; i < NA * ld; i += nthr) L[i] = 0.f;
  }
  __syncthreads();
  // ---- residual (FP64): R = -(A_H c + alpha t + P^T w (f(U) - g), t.c + alpha s + u~.w (f(U) - g)),
  // by the threads t0, t0 + stride, ...; the last warp also forms the alpha row
  const double alpha = S.sa[1];
  const double sig = A.sigma_H;
  auto form_residual = [&](int t0, int stride) {
    for (int p = t0; p < NH; p += stride) {
      int z[3];
      unknown_coords<D>(p, A.nc, z);
      const double ahc = coarse_apply<D>(A, S.c, coarse_offset<D>(z, A.nc), z);
      rf[p] = (float)(-(ahc + alpha * S.t[p] + node_channel<D, true>(cellsum, A.nc, z, G::RA)));
    }
    if (tid >= nthr - 32) {
      double s2 = 0.0, tc = 0.0;
      for (int c = lane; c < ncell; c += 32) s2 += cellsum[(long long)c * G::NVAL + G::SA];
      for (int p = lane; p < NH; p += 32) {
        int z[3];
        unknown_coords<D>(p, A.nc, z);
        tc += S.t[p] * S.c[coarse_offset<D>(z, A.nc)];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        tc += __shfl_xor_sync(0xffffffffu, tc, o);
      }
      if (lane == 0) rf[NH] = (float)(-(tc + alpha * S.sa[0] + s2));
    }
  };
  int dropped = 0;
  bool ok = true;
  const float* Xuse = L;   // the kept inverse (chord steps)
  if (!first) {
    form_residual(tid, nthr);
    __syncthreads();
  } else {
    // the Jacobian (fixed point: the Galerkin stiffness) in FP32 from the FP32 channels: the
    // lower band (neighbours q <= p of unknown p in the 3^d box), the border row and the corner,
    // an entry per thread
    const float sigf = (float)sig;
    const int4* jt = reinterpret_cast<const int4*>(A.jtab);
    for (int e = tid; e < NH * (N3 + 1); e += nthr) {
      int w[kJW<D>];
#pragma unroll
      for (int i = 0; i < kJW<D> / 4; ++i) {
        const int4 t4 = __ldg(jt + (size_t)e * (kJW<D> / 4) + i);
        w[4 * i] = t4.x;
        w[4 * i + 1] = t4.y;
        w[4 * i + 2] = t4.z;
        w[4 * i + 3] = t4.w;
      }
      if (w[0] < 0) continue;
      float x = 0.f;
      if (!fixedp) {
#pragma unroll
        for (int o = 0; o < G::NV; ++o)
          if (w[2 + o] >= 0) x += reinterpret_cast<const float*>(cellsum + w[2 + o])[0];
      }
      const int p = (w[1] >> 8) & 255;
      if (w[1] & 4) {
        L[w[0]] = (float)S.t[p] + x;
        continue;
      }
      const int dist = w[1] & 3;
      if (A.vc.a64) {
        int z[3], dv[3], r2 = (w[1] >> 16) & 255;
        unknown_coords<D>(p, A.nc, z);
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
          dv[ax] = r2 % 3 - 1;
          r2 /= 3;
        }
        x += (float)coarse_stiffness<D>(A, z, dv, dist);
      } else {
        if (dist == 0) x += sigf * (float)(2 * D);
        else if (dist == 1) x -= sigf;
      }
      L[w[0]] = x;
    }
    if (tid == 0) L[NH * ld + NH] = (float)S.sa[0] + (fixedp ? 0.f : s3_sh);
    __syncthreads();
    // ---- band LDL^T of J on warp 0 while the other warps form the residual, then the inverse,
    // a column per thread
    const int band = aug_band<D>(A.nc);
    float* rd = L + (size_t)NA * ld;
    if (tid < 32) {
      int dr = 0;
      bool okw;
      // the benchmark shapes with their size and band fixed at compile time
      if (D == 2 && NA == 50 && band == 8)
        okw = ldlt_band_warp_ns<float, 2, 50, 8>(L, NA, ld, rd, band, 1, true, 1e-6, &dr);
      else if (D == 2 && NA == 10 && band == 4)
        okw = ldlt_band_warp_ns<float, 1, 10, 4>(L, NA, ld, rd, band, 1, true, 1e-6, &dr);
      else if (D == 3 && NA == 28 && band == 13)
        okw = ldlt_band_warp_ns<float, 4, 28, 13>(L, NA, ld, rd, band, 1, true, 1e-6, &dr);
      else
        okw = ldlt_band_warp<float>(L, NA, ld, rd, band, 1, true, 1e-6, &dr);
      if (tid == 0) {
        fac_sh[0] = okw ? 1 : 0;
        fac_sh[1] = dr;
      }
    } else {
      form_residual(tid - 32, nthr - 32);
    }
    __syncthreads();
    ok = fac_sh[0] != 0;
    dropped = fac_sh[1];
    if (tid < NA) band_inverse_dispatch<D>(L, rd, NA, ld, band, tid, X);
    __syncthreads();
    // keep J^{-1} where the factor was (the factor is no longer needed)
    for (int i = tid; i < NA * ld; i += nthr) L[i] = X[i];
    Xuse = X;
  }
  // ---- the step y = J^{-1} R, then (c, alpha) += y and the convergence test
  small_matvec(Xuse, NA, ld, rf, dl);
  __syncthreads();
  newton_update_mixed<D>(A, dl, NH, S, dropped, ok, writer, red_sh);
}

// After a pass, in every block: cell sums, the dense system, the Newton step, convergence.
// In the mixed path (JF32) the first iteration factors its Jacobian into L (LDL^T, FP32, with
// the reciprocal pivots after it) and the later iterations are chord steps with that factor.
// The fixed-point iteration (A.fixed_point) factors the Galerkin stiffness [[A_H, t], [t^T, s]]
// once, in the path's precision, and every iteration solves with it against the residual
// (y_{k+1} = y_k - K^{-1} R(y_k), i.e. K y_{k+1} = G - B^T W f(B y_k)).  `partials` holds this
// iteration's sums, one row per coarse cell; only the writer block reports to DevState.
// Not inlined: the dense step runs once per pass, and its own register allocation keeps it
// from raising the pressure in the fine pass.
template <int D, bool JF32>
__device__ __noinline__ void newton_step(const AugArgs& A, const double* __restrict__ partials, double* cellsum,
                                         double* M,
                            double* R, typename std::conditional<JF32, float, double>::type* L, const StepState& S,
                            bool first, bool writer) {
  using FT = typename std::conditional<JF32, float, double>::type;
  using G = Aug<D, JF32>;
  const int tid = threadIdx.x;
  const int ncell = (int)ipow(A.nc, D);
  const int NH = (int)ipow(A.nc - 1, D);
  const int NA = NH + 1;
  const int ld = NA + 1;
  constexpr int N3 = D == 2 ? 9 : 27;
  if constexpr (JF32) {
    newton_step_mixed<D>(A, partials, cellsum, M, R, L, S, first, writer);
    return;
  }
  const double alpha = S.sa[1];
  const double* t_vec = S.t;
  if ((JF32 || A.fixed_point) && !first) {
    // chord / fixed-point step: the residual at the new iterate (mixed path: first-pass FP64
    // sums plus this pass's increments; FP64 path: this pass's sums), solved with the factor
    // of the first iteration
    const int total = ncell * (G::NV + 1);
    for (int base = tid; base < total; base += 4 * blockDim.x) {
      double x[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int idx = base + r * blockDim.x;
        x[r] = 0.0;
        if (idx < total) {
          const int cell = idx / (G::NV + 1), v = idx % (G::NV + 1);
          const int chn = v < G::NV ? G::RA + v : G::SA;
          x[r] = __ldcg(partials + (size_t)cell * G::NVAL + chn);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int idx = base + r * blockDim.x;
        if (idx < total) {
          const int cell = idx / (G::NV + 1), v = idx % (G::NV + 1);
          const int chn = v < G::NV ? G::RA + v : G::SA;
          cellsum[(size_t)cell * G::NVAL + chn] = JF32 ? x[r] + S.basev[idx] : x[r];
        }
      }
    }
    __syncthreads();
    for (int p = tid; p < NH; p += blockDim.x) {
      int z[3];
      unknown_coords<D>(p, A.nc, z);
      const double ahc = coarse_apply<D>(A, S.c, coarse_offset<D>(z, A.nc), z);
      R[p] = -(ahc + alpha * t_vec[p] + node_channel<D, JF32>(cellsum, A.nc, z, G::RA));
    }
    if (tid < 32) {
      double s2 = 0.0, tc = 0.0;
      for (int c = tid; c < ncell; c += 32) s2 += cellsum[(long long)c * G::NVAL + G::SA];
      for (int p = tid; p < NH; p += 32) {
        int z[3];
        unknown_coords<D>(p, A.nc, z);
        tc += t_vec[p] * S.c[coarse_offset<D>(z, A.nc)];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        tc += __shfl_xor_sync(0xffffffffu, tc, o);
      }
      if (tid == 0) R[NH] = -(tc + alpha * S.sa[0] + s2);
    }
    __syncthreads();
    if (tid < 32) ldlt_solve_band_warp<FT>(L, NA, ld, L + (size_t)NA * ld, aug_band<D>(A.nc), 1, R);
    __syncthreads();
    newton_update<D>(A, R, NH, S, 0, true, writer);
    return;
  }
  // the cell sums (one row per coarse cell), eight loaded together
  auto needed = [&](int v) { return !((!first && v >= G::TT && v < G::JB) || (A.fixed_point && v >= G::JB)); };
  {
    const int total = ncell * G::NVAL;
    for (int base = tid; base < total; base += 8 * blockDim.x) {
      double x[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int idx = base + r * blockDim.x;
        x[r] = (idx < total && needed(idx % G::NVAL)) ? __ldcg(partials + idx) : 0.0;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int idx = base + r * blockDim.x;
        if (idx < total && needed(idx % G::NVAL)) cellsum[idx] = x[r];
      }
    }
  }
  for (int idx = tid; idx < NA * ld; idx += blockDim.x) M[idx] = 0.0;
  __syncthreads();
  if (JF32) {
    // mixed path: after the first pass the residual channels hold increments; the first
    // pass's FP64 sums are kept in basev and added back (fixed order, same thread each time)
    for (int idx = tid; idx < ncell * (G::NV + 1); idx += blockDim.x) {
      const int cell = idx / (G::NV + 1), v = idx % (G::NV + 1);
      const long long ch = (long long)cell * G::NVAL + (v < G::NV ? G::RA + v : G::SA);
      if (first)
        S.basev[idx] = cellsum[ch];
      else
        cellsum[ch] += S.basev[idx];
    }
    __syncthreads();
  }
  if (first) {
    for (int p = tid; p < NH; p += blockDim.x) {
      int z[3];
      unknown_coords<D>(p, A.nc, z);
      S.t[p] = node_channel<D, JF32>(cellsum, A.nc, z, G::TT);
    }
    if (tid < 32) {
      double s0 = 0.0;
      for (int c = tid; c < ncell; c += 32) s0 += cellsum[(long long)c * G::NVAL + G::SS];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      if (tid == 0) S.sa[0] = s0;
    }
    __syncthreads();
  }
  // J_HH on the coarse-edge pattern (entries for every neighbour in the 3^d box)
  for (int idx = tid; idx < NH * N3; idx += blockDim.x) {
    const int p = idx / N3;
    int r = idx % N3;
    int z[3], zq[3], dv[3];
    unknown_coords<D>(p, A.nc, z);
    bool ok = true;
    int q = 0, mul = 1, dist = 0;
    for (int ax = 0; ax < D; ++ax) {
      const int d = r % 3 - 1;
      r /= 3;
      dv[ax] = d;
      zq[ax] = z[ax] + d;
      if (zq[ax] < 1 || zq[ax] > A.nc - 1) ok = false;
      q += (zq[ax] - 1) * mul;
      mul *= (A.nc - 1);
      dist += abs(d);
    }
    if (!ok) continue;
    double v = A.fixed_point ? 0.0 : pair_channel<D, JF32>(cellsum, A.nc, z, zq);
    v += coarse_stiffness<D>(A, z, dv, dist);
    M[p * ld + q] = v;
  }
  // residual and the alpha border
  for (int p = tid; p < NH; p += blockDim.x) {
    int z[3];
    unknown_coords<D>(p, A.nc, z);
    const double ahc = coarse_apply<D>(A, S.c, coarse_offset<D>(z, A.nc), z);
    R[p] = -(ahc + alpha * t_vec[p] + node_channel<D, JF32>(cellsum, A.nc, z, G::RA));
    const double jb = t_vec[p] + (A.fixed_point ? 0.0 : node_channel<D, JF32>(cellsum, A.nc, z, G::JB));
    M[p * ld + NH] = jb;
    M[NH * ld + p] = jb;
  }
  if (tid < 32) {
    double s2 = 0.0, s3 = 0.0, tc = 0.0;
    for (int c = tid; c < ncell; c += 32) {
      s2 += cellsum[(long long)c * G::NVAL + G::SA];
      if (!A.fixed_point) s3 += cellsum[(long long)c * G::NVAL + G::JS];
    }
    for (int p = tid; p < NH; p += 32) {
      int z[3];
      unknown_coords<D>(p, A.nc, z);
      tc += t_vec[p] * S.c[coarse_offset<D>(z, A.nc)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      tc += __shfl_xor_sync(0xffffffffu, tc, o);
    }
    if (tid == 0) {
      R[NH] = -(tc + alpha * S.sa[0] + s2);
      M[NH * ld + NH] = S.sa[0] + s3;
    }
  }
  __syncthreads();
  // Newton step on warp 0.  FP64 path: LDL^T in FP64.  Mixed path: LDL^T in FP32, kept in L
  // for the chord steps of the later iterations.
  int dropped = 0;
  bool ok = true;
  for (int idx = tid; idx < NA * ld; idx += blockDim.x) L[idx] = (FT)M[idx];
  __syncthreads();
  const int band = aug_band<D>(A.nc);
  FT* rd = L + (size_t)NA * ld;
  if (tid < 32) {
    ok = ldlt_band_warp<FT>(L, NA, ld, rd, band, 1, true, JF32 ? 1e-6 : 1e-14, &dropped);
    ldlt_solve_band_warp<FT>(L, NA, ld, rd, band, 1, R);
  }
  __syncthreads();
  newton_update<D>(A, R, NH, S, dropped, ok, writer);
}

// (c, alpha) += the step in R, convergence test and stop flags (warp 0 of every block; the
// writer block also reports to DevState).
template <int D>
__device__ void newton_update(const AugArgs& A, const double* R, int NH, const StepState& S, int dropped, bool ok,
                              bool writer) {
  const int tid = threadIdx.x;
  if (tid < 32) {
    double dmax = 0.0, ymax = 0.0;
    bool finite = true;
    for (int p = tid; p < NH; p += 32) {
      int z[3];
      unknown_coords<D>(p, A.nc, z);
      const long long off = coarse_offset<D>(z, A.nc);
      const double nv = S.c[off] + R[p];
      if (!isfinite(nv)) finite = false;
      S.c[off] = nv;
      dmax = fmax(dmax, fabs(R[p]));
      ymax = fmax(ymax, fabs(nv));
    }
    const double na = S.sa[1] + R[NH];
    if (tid == 0) {
      if (!isfinite(na)) finite = false;
      dmax = fmax(dmax, fabs(R[NH]));
      ymax = fmax(ymax, fabs(na));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      ymax = fmax(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    }
    finite = __all_sync(0xffffffffu, finite);
    if (tid == 0) {
      S.sa[1] = na;
      S.flags[1] = (!ok || !finite) ? 1 : 0;
      S.flags[0] = (dmax <= A.tol * fmax(1.0, ymax)) ? 1 : 0;
      if (writer) {
        if (dropped) atomicOr(&A.st->flags, kFlagDropped);
        if (!ok) atomicOr(&A.st->flags, kFlagNotSPD);
        if (!finite) atomicOr(&A.st->flags, kFlagNonfinite);
      }
    }
  }
}

// Before the first pass, in every block: c = 0, alpha = 1, flags clear.
template <int D>
__device__ void step_state_init(const AugArgs& A, const StepState& S) {
  const long long cn = ipow(A.nc + 1, D);
  for (long long i = threadIdx.x; i < cn; i += blockDim.x) S.c[i] = 0.0;
  if (threadIdx.x == 0) {
    S.sa[1] = 1.0;
    S.flags[0] = 0;
    S.flags[1] = 0;
  }
  __syncthreads();
}

// After the iteration, the writer block: iteration count, alpha and the Newton-cap flag.
__device__ void step_report(const AugArgs& A, const StepState& S, int it, bool writer) {
  if (writer && threadIdx.x == 0) {
    if (!(S.flags[0] && !S.flags[1])) atomicOr(&A.st->flags, kFlagNewtonCap);
    A.st->newton_iters[A.level_index] += it > A.maxit ? A.maxit : it;
    A.st->alpha[A.level_index] = S.sa[1];
  }
}

// VC: the first pass forms A_k u~ with the coefficient's edge weights (a variant of its own, so
// that the constant-coefficient kernels keep their register allocation).
template <int D, bool JF32, bool VC>
__global__ void __launch_bounds__(Aug<D, JF32>::NT, 512 / Aug<D, JF32>::NT) k_augmented(AugArgs A) {
  pdl_start();
  using G = Aug<D, JF32>;
  using FT = typename std::conditional<JF32, float, double>::type;
  extern __shared__ double sm[];
  double* acc = sm;                                 // channel rows [NVAL][NT]
  __shared__ double cv[G::NV];
  __shared__ int flags_sh[2];
  __shared__ int stop;
  __shared__ int last_sh;
  const int tid = threadIdx.x;
  const unsigned nblocks = gridDim.x;
  const int cell = blockIdx.x / A.bpc;
  const int bic = blockIdx.x % A.bpc;
  const int ncell = (int)ipow(A.nc, D);
  const int NA = (int)ipow(A.nc - 1, D) + 1;
  int cellc[3] = {0, 0, 0};
  {
    int t = cell;
    for (int q = 0; q < D; ++q) {
      cellc[q] = t % A.nc;
      t /= A.nc;
    }
  }
  long long vert_off = 0;   // coarse nodal offset of this thread's cell vertex (tid < NV)
  if (tid < G::NV) {
    long long mul = 1;
    for (int q = 0; q < D; ++q) {
      vert_off += (long long)(cellc[q] + ((tid >> q) & 1)) * mul;
      mul *= (A.nc + 1);
    }
  }
  double* cellsum = acc;
  double* M = cellsum + (size_t)ncell * G::NVAL;
  double* R = M + (size_t)NA * (NA + 1);
  StepState S;
  FT* L;
  AugSmem<D, JF32>::carve(sm, A.nc, S, L);
  S.flags = flags_sh;
  step_state_init<D>(A, S);
  const bool writer = blockIdx.x == 0;
  int it = 0;
  for (it = 1; it <= A.maxit; ++it) {
    const bool first = it == 1;
    // partial rows alternate between two buffers: a block that starts the next pass cannot
    // overwrite sums that another block is still reading
    double* pbuf = A.partials + (size_t)(it & 1) * A.pstride;
    if (tid < G::NV) cv[tid] = S.c[vert_off];
    if (tid == 0) stop = ((volatile int*)&A.st->abort)[0];
    // chord steps of the mixed path fill the residual channels RA, SA only
    Rows<D, JF32>::zero(acc, first, A.fixed_point != 0, tid);
    __syncthreads();
    if (stop) break;
    fine_pass<D, JF32, VC>(A, first ? kFirst : kNewton, acc, cv, S.sa[1], cell, bic);
    block_reduce_rows<D, JF32>(A, acc, pbuf + (size_t)blockIdx.x * G::NVAL, first, A.fixed_point != 0);
    // one row per cell for the dense step: with one block per cell its partial row, else the
    // cell sums of this iteration's buffer (formed by the cell's last block)
    const double* rows = pbuf;
    if (A.bpc > 1) {
      double* cbuf = A.partials + 2 * A.pstride + (size_t)(it & 1) * ncell * G::NVAL;
      cell_reduce<D, JF32>(A, pbuf, cbuf, cell, first, &last_sh);
      rows = cbuf;
    }
    grid_barrier(A.st, nblocks, A.bar_spins, first && (int)blockIdx.x == A.bar_skip);
    newton_step<D, JF32>(A, rows, cellsum, M, R, L, S, first, writer);
    __syncthreads();
    if (flags_sh[0] || flags_sh[1]) break;
  }
  step_report(A, S, it, writer);
  if (flags_sh[1] && writer && tid == 0) A.st->abort = 1;
  if (A.split_update) {
    // the update runs as a kernel of its own: block 0 hands over c and alpha - 1 in FP32 (the
    // update forms the increment (alpha - 1) u~ + P c in FP32)
    if (blockIdx.x == 0) {
      float* cf = reinterpret_cast<float*>(A.cfin);
      const int cn = (int)ipow(A.nc + 1, D);
      for (int i = tid; i < cn; i += blockDim.x) cf[i] = (float)S.c[i];
      if (tid == 0) cf[cn] = (float)(S.sa[1] - 1.0);
    }
    return;
  }
  // final update u = alpha u~ + P_{H->k} c
  if (tid < G::NV) cv[tid] = S.c[vert_off];
  __syncthreads();
  fine_pass<D, JF32, VC>(A, kUpdate, acc, cv, S.sa[1], cell, bic);
}

// The final update of a correction step's mixed path, u = alpha u~ + P_{H->k} c, as a
// node-parallel kernel at full occupancy (the largest levels, where the Newton kernel's own pass
// at its 16 warps per SM is latency-bound).  Node (x, y[, z]) lies in coarse cell x >> ls (s =
// 2^ls fine cells per coarse cell) at offsets o = x & (s-1); sorting the offsets in decreasing
// order (ties: x before y before z) gives the Kuhn simplex v_0 = 0, v_{t+1} = v_t + e_{pi_t}
// with barycentric weights lambda_0 = (s - o_{pi_0})/s, lambda_t = (o_{pi_{t-1}} - o_{pi_t})/s,
// lambda_d = o_{pi_{d-1}}/s -- the simplices and weights of the column walk.  The increment
// (alpha - 1) u~ + P c is formed in FP32 from the FP32 coarse values the Newton kernel left in
// cf (then alpha - 1) and added to the float-float u~; the result is float-float, or FP64 for
// the solve's last step (out_f64).  Threads run along x; each block walks rows y (and z) with
// the grid's row stride, so the coarse values are staged once per block.
template <int D>
__global__ void __launch_bounds__(256) k_aug_update(double* __restrict__ u, int n, int ls, int nc,
                                                    const float* __restrict__ cf, int out_f64) {
  pdl_start();
  __shared__ float cs[128];
  __shared__ float am1;
  const int cn = (int)ipow(nc + 1, D);
  for (int i = threadIdx.x; i < cn; i += blockDim.x) cs[i] = cf[i];
  if (threadIdx.x == 0) am1 = cf[cn];
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < 1 || x >= n) return;
  const long long np = n + 1;
  const int s = 1 << ls;
  const float inv_s = 1.0f / (float)s;
  const int cp = nc + 1;
  const int ox = x & (s - 1), cx = x >> ls;
  const long long rows = D == 2 ? (long long)(n - 1) : (long long)(n - 1) * (n - 1);
  for (long long r = blockIdx.y; r < rows; r += gridDim.y) {
    const int y = (int)(D == 2 ? r : r % (n - 1)) + 1;
    const int z = D == 3 ? (int)(r / (n - 1)) + 1 : 0;
    const long long idx = (D == 2 ? (long long)y : (long long)z * np + y) * np + x;
    const int o[3] = {ox, y & (s - 1), D == 3 ? (z & (s - 1)) : 0};
    const int cc[3] = {cx, y >> ls, D == 3 ? (z >> ls) : 0};
    // axes in decreasing offset order, ties to the lower axis
    int pi[3] = {0, 1, 2};
    if (D == 2) {
      if (o[1] > o[0]) {
        pi[0] = 1;
        pi[1] = 0;
      }
    } else {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2 - a; ++b)
          if (o[pi[b + 1]] > o[pi[b]]) {
            const int t = pi[b];
            pi[b] = pi[b + 1];
            pi[b + 1] = t;
          }
    }
    int vo[3] = {0, 0, 0};   // the current simplex vertex, coarse offsets
    auto cval = [&]() {
      const int base = D == 2 ? (cc[1] + vo[1]) * cp + cc[0] + vo[0]
                              : ((cc[2] + vo[2]) * cp + cc[1] + vo[1]) * cp + cc[0] + vo[0];
      return cs[base];
    };
    float pc = (float)(s - o[pi[0]]) * cval();
#pragma unroll
    for (int t = 0; t < D; ++t) {
      vo[pi[t]] = 1;
      const int w = t + 1 < D ? o[pi[t]] - o[pi[t + 1]] : o[pi[t]];
      pc = fmaf((float)w, cval(), pc);
    }
    pc *= inv_s;
    const ff ut = ff_load(u + idx);
    const ff un = ff_add_f(ut, fmaf(am1, ut.hi, pc));
    if (out_f64)
      u[idx] = (y & 1) ? ff_to_double_rn(un) : ff_to_double_fast(un);
    else
      ff_store(u + idx, un);
  }
}

template <int D, bool JF32>
__device__ __forceinline__ void k_augmented_cluster_body(const AugArgs& A) {
  using G = Aug<D, JF32>;
  using FT = typename std::conditional<JF32, float, double>::type;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int CS = (int)cluster.num_blocks();
  extern __shared__ double sm[];
  double* acc = sm;
  __shared__ double cv[G::NV];
  __shared__ int flags_sh[2];
  __shared__ int stop;
  const int tid = threadIdx.x;
  const int ncell = (int)ipow(A.nc, D);
  const int NA = (int)ipow(A.nc - 1, D) + 1;
  double* cellsum = acc;
  double* M = cellsum + (size_t)ncell * G::NVAL;
  double* R = M + (size_t)NA * (NA + 1);
  StepState S;
  FT* L;
  AugSmem<D, JF32>::carve(sm, A.nc, S, L);
  S.flags = flags_sh;
  auto vertex_offset = [&](int cell, int v) {
    long long off = 0, mul = 1;
    int t = cell;
    for (int q = 0; q < D; ++q) {
      off += (long long)(t % A.nc + ((v >> q) & 1)) * mul;
      t /= A.nc;
      mul *= (A.nc + 1);
    }
    return off;
  };
  step_state_init<D>(A, S);
  const bool writer = rank == 0;
  int it = 0;
  for (it = 1; it <= A.maxit; ++it) {
    const bool first = it == 1;
    double* pbuf = A.partials + (size_t)(it & 1) * A.pstride;
    if (tid == 0) stop = ((volatile int*)&A.st->abort)[0];
    __syncthreads();
    if (stop) break;
    for (int cell = rank; cell < ncell; cell += CS) {
      if (tid < G::NV) cv[tid] = S.c[vertex_offset(cell, tid)];
      Rows<D, JF32>::zero(acc, first, A.fixed_point != 0, tid);
      __syncthreads();
      fine_pass<D, JF32>(A, first ? kFirst : kNewton, acc, cv, S.sa[1], cell, 0);
      block_reduce_rows<D, JF32>(A, acc, pbuf + (size_t)cell * G::NVAL, first, A.fixed_point != 0);
    }
    cluster.sync();
    newton_step<D, JF32>(A, pbuf, cellsum, M, R, L, S, first, writer);
    __syncthreads();
    if (flags_sh[0] || flags_sh[1]) break;
  }
  step_report(A, S, it, writer);
  if (flags_sh[1] && writer && tid == 0) A.st->abort = 1;
  for (int cell = rank; cell < ncell; cell += CS) {
    if (tid < G::NV) cv[tid] = S.c[vertex_offset(cell, tid)];
    __syncthreads();
    fine_pass<D, JF32>(A, kUpdate, acc, cv, S.sa[1], cell, 0);
    __syncthreads();
  }
}

template <int D, bool JF32>
__global__ void __launch_bounds__(Aug<D, JF32>::NT, 512 / Aug<D, JF32>::NT) k_augmented_cluster(const __grid_constant__ AugArgs A) {
  pdl_start();
  k_augmented_cluster_body<D, JF32>(A);
}

template <int D, bool JF32>
size_t aug_smem(int nc) {
  return AugSmem<D, JF32>::bytes(nc);
}

// Blocks per SM of the cooperative kernel of one precision when launched with `smem` dynamic
// bytes (the smaller of its constant- and variable-coefficient variants).
template <int D, bool JF32>
int aug_occupancy(size_t smem) {
  int occ = 0, occ_vc = 0;
  raise_dyn_smem((const void*)k_augmented<D, JF32, false>, smem);
  raise_dyn_smem((const void*)k_augmented<D, JF32, true>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_augmented<D, JF32, false>, Aug<D, JF32>::NT, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_vc, k_augmented<D, JF32, true>, Aug<D, JF32>::NT, smem);
  return occ < occ_vc ? occ : occ_vc;
}

}  // namespace

// ============================================================================ launchers

cudaError_t launch_coarse_inverse(int dim, LevelGeo g1, double* Ainv, DevState* st, cudaStream_t s,
                                  const VarCoef* vc) {
  const int m = g1.n - 1;
  const int N = (int)ipow(m, dim);
  const size_t smem = sizeof(double) * ((size_t)N * (N + 1) + 3 * N + 4);
  cudaError_t e = raise_dyn_smem((const void*)k_coarse_inverse, smem);
  if (e != cudaSuccess) return e;
  launch_k(k_coarse_inverse, 1, 64, smem, s, dim, g1.n, Ainv, st, vc ? *vc : VarCoef{});
  return cudaGetLastError();
}

cudaError_t launch_level1_newton(int dim, LevelGeo g1, const double* gn, double* u, int kind, double a, double tol,
                                 int maxit, bool f32_factor, DevState* st, cudaStream_t s, bool out_ff,
                                 const VarCoef* vc) {
  const VarCoef v = vc ? *vc : VarCoef{};
  const int m = g1.n - 1;
  const size_t N = (size_t)ipow(m, dim);
  cudaError_t e;
  if (f32_factor) {
    const size_t smem = sizeof(double) * (3 * N + 2) + sizeof(float) * (N * (N + 1) + 2 * N + 4);
    if ((e = raise_dyn_smem((const void*)k_level1_newton<float>, smem)) != cudaSuccess) return e;
    launch_k(k_level1_newton<float>, 1, 256, smem, s, dim, g1.n, gn, u, kind, a, tol, maxit, st, out_ff ? 1 : 0, v);
  } else {
    const size_t smem = sizeof(double) * (3 * N + 2 + N * (N + 1) + 2 * N + 4);
    if ((e = raise_dyn_smem((const void*)k_level1_newton<double>, smem)) != cudaSuccess) return e;
    launch_k(k_level1_newton<double>, 1, 256, smem, s, dim, g1.n, gn, u, kind, a, tol, maxit, st, out_ff ? 1 : 0, v);
  }
  return cudaGetLastError();
}

int aug_nvals(int dim) { return dim == 2 ? Aug<2, false>::NVAL : Aug<3, false>::NVAL; }

size_t aug_jtab_ints(int dim, int coarse_cells) {
  return dim == 2 ? (size_t)aug_jtab_entries<2>(coarse_cells) * kJW<2>
                  : (size_t)aug_jtab_entries<3>(coarse_cells) * kJW<3>;
}

cudaError_t launch_aug_jtab(int dim, int coarse_cells, int* tab, cudaStream_t s) {
  if (dim == 2)
    launch_k(k_aug_jtab<2>, 4, 256, 0, s, coarse_cells, tab);
  else
    launch_k(k_aug_jtab<3>, 4, 256, 0, s, coarse_cells, tab);
  return cudaGetLastError();
}

void aug_configure(int dim, int coarse_cells, bool mixed, AugBuffers* ab) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    sms = 0;
  const int ncell = (int)ipow(coarse_cells, dim);
  // the context's precision picks the kernel: its shared memory and residency set the grid
  const size_t smem = mixed ? (dim == 2 ? aug_smem<2, true>(coarse_cells) : aug_smem<3, true>(coarse_cells))
                            : (dim == 2 ? aug_smem<2, false>(coarse_cells) : aug_smem<3, false>(coarse_cells));
  int occ_min = 0;
  if (sms > 0) {
    if (dim == 2)
      occ_min = mixed ? aug_occupancy<2, true>(smem) : aug_occupancy<2, false>(smem);
    else
      occ_min = mixed ? aug_occupancy<3, true>(smem) : aug_occupancy<3, false>(smem);
  }
  // at most 16 warps per SM (two 2D blocks, four 3D ones): every block takes the dense Newton
  // step, so more blocks per SM add contending copies of it and more partial rows to gather,
  // while the passes do not speed up (FP64 path: bound by the SM's FP64 pipe); the 2D FP64
  // solve measured 20 % slower at three blocks (24 warps) than at two
  const int nt = dim == 2 ? Aug<2, false>::NT : Aug<3, false>::NT;
  if (occ_min > 512 / nt) occ_min = 512 / nt;
  int bpc = sms > 0 ? (occ_min * sms) / ncell : 1;
  if (bpc < 0) bpc = 0;
  ab->bpc = bpc;
  ab->smem = smem;
  ab->sms = sms;
  ab->nt = dim == 2 ? Aug<2, false>::NT : Aug<3, false>::NT;
  ab->partial_items = (size_t)ncell * (bpc > 0 ? bpc : 1);
}

template <int D, bool JF32>
int cluster_size_for(int ncell, size_t smem) {
  const int nt = Aug<D, JF32>::NT;
  raise_dyn_smem((const void*)k_augmented_cluster<D, JF32>, smem);
  cudaFuncSetAttribute(k_augmented_cluster<D, JF32>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int cs = ncell < 16 ? ncell : 16; cs >= 1; cs >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_augmented_cluster<D, JF32>, &cfg) == cudaSuccess && n > 0) return cs;
  }
  cudaGetLastError();
  return 0;
}

int aug_cluster_size(int dim, int coarse_cells, bool jac_f32, size_t smem) {
  const int ncell = (int)ipow(coarse_cells, dim);
  if (dim == 2) return jac_f32 ? cluster_size_for<2, true>(ncell, smem) : cluster_size_for<2, false>(ncell, smem);
  return jac_f32 ? cluster_size_for<3, true>(ncell, smem) : cluster_size_for<3, false>(ncell, smem);
}

// Launch shapes of the cooperative augmented kernel picked by the autotuner
// (fmg_autotune_augmented), per device, dimension, 1/H, level and precision; absent entries use
// the rule of aug_shape.
namespace {
std::mutex g_aug_mu;
std::map<std::tuple<int, int, int, int, int>, AugShape> g_aug_shapes;
std::tuple<int, int, int, int, int> aug_key(int dim, int nc, int level, bool mixed) {
  int dev = 0;
  cudaGetDevice(&dev);
  return std::make_tuple(dev, dim, nc, level, mixed ? 1 : 0);
}
}  // namespace

void set_aug_shape(int dim, int coarse_cells, int level, bool mixed, AugShape sh) {
  std::lock_guard<std::mutex> lk(g_aug_mu);
  g_aug_shapes[aug_key(dim, coarse_cells, level, mixed)] = sh;
}

bool aug_shape_tuned(int dim, int coarse_cells, int level, bool mixed, AugShape* out) {
  std::lock_guard<std::mutex> lk(g_aug_mu);
  auto it = g_aug_shapes.find(aug_key(dim, coarse_cells, level, mixed));
  if (it == g_aug_shapes.end()) return false;
  if (out) *out = it->second;
  return true;
}

AugShape aug_shape(int dim, int coarse_cells, int level, bool jac_f32, const AugBuffers& ab, bool tuned) {
  const int ncell = (int)ipow(coarse_cells, dim);
  const int sfine = 1 << (level - 1);
  const int nt = ab.nt;
  // column chunks of up to 32 nodes; on smaller levels shorter ones, until every thread has
  // an item (each chunk costs one moment-to-channel conversion, so they are no shorter than
  // that needs, and at least 2 nodes long).  FP64 path: every co-resident thread of the
  // grid, since its per-node work is FP64 and one SM sub-partition issues one FP64 warp
  // instruction per ~64 clocks.  Mixed path (FP32 float-float work per node): the threads of
  // one block per cell, and only as many blocks as the chunks fill -- on small levels one
  // per cell, which keeps the partial rows every block gathers and the arrivals at each grid
  // barrier few.
  const long long ncol = ipow(sfine, dim - 1);
  const long long target = (long long)(jac_f32 ? 1 : ab.bpc) * nt * ncell;
  int chunk = sfine < 32 ? sfine : 32;
  while (chunk > 2 && ncol * (sfine / chunk) * ncell < target) chunk >>= 1;
  const long long items = ncol * (sfine / chunk);
  // blocks per cell: about one chunk per thread; on the FP64 path, when that leaves blocks
  // unfilled, the chunks are spread over all co-resident blocks of the cell instead
  int bpc = (int)((items + nt - 1) / nt);
  if (jac_f32) {
    if (bpc > ab.bpc) bpc = ab.bpc;
  } else if (bpc > ab.bpc || items < (long long)ab.bpc * nt) {
    bpc = (int)(items < ab.bpc ? items : ab.bpc);
  }
  if (bpc < 1) bpc = 1;
  AugShape sh{chunk, bpc};
  AugShape t;
  if (tuned && aug_shape_tuned(dim, coarse_cells, level, jac_f32, &t)) {
    // a tuned shape within the launch's limits: a power-of-two chunk that divides the column,
    // at most the co-resident blocks per cell that the partial rows are sized for
    if (t.chunk >= 2 && t.chunk <= 32 && t.chunk <= sfine && (t.chunk & (t.chunk - 1)) == 0) sh.chunk = t.chunk;
    if (t.bpc >= 1 && t.bpc <= ab.bpc) sh.bpc = t.bpc;
  }
  return sh;
}

cudaError_t launch_augmented(int dim, int coarse_cells, int level, LevelGeo gk, double* u, const double* gn,
                             int kind, double a, double tol, int maxit, bool jac_f32, const AugBuffers& ab,
                             DevState* st, int level_index, cudaStream_t s, int cluster_size, int fixed_point,
                             int out_f64, const VarCoef* vc) {
  const size_t smem = ab.smem;
  const int nt = ab.nt;
  if (ab.bpc < 1 || nt < 1) return cudaErrorInvalidConfiguration;
  const int ncell = (int)ipow(coarse_cells, dim);
  const int sfine = 1 << (level - 1);
  // the cluster variant (one block per cell in turn) takes the rule's chunks, never a tuned shape
  const AugShape shape = aug_shape(dim, coarse_cells, level, jac_f32, ab, cluster_size == 0);
  int chunk = shape.chunk, bpc = shape.bpc;
  AugArgs A;
  A.dim = dim;
  A.nc = coarse_cells;
  A.s = sfine;
  A.ls = level - 1;
  A.n = gk.n;
  A.kind = kind;
  A.maxit = maxit;
  A.level_index = level_index;
  A.fixed_point = fixed_point;
  A.out_f64 = out_f64;
  A.bpc = bpc;
  A.chunk = chunk;
  A.a = a;
  const double h = 1.0 / gk.n;
  A.w = dim == 2 ? h * h : h * h * h;
  A.sigma_k = dim == 2 ? 1.0 : h;
  A.sigma_H = dim == 2 ? 1.0 : 1.0 / coarse_cells;
  A.tol = tol;
  A.a_ff = ff_from_double(a);
  A.sigma_ff = ff_from_double(A.sigma_k);
  A.u = u;
  A.g = gn;
  A.partials = ab.partials;
  A.pstride = (long long)ab.partial_items * (dim == 2 ? Aug<2, false>::NVAL : Aug<3, false>::NVAL);
  A.Ainv = ab.Ainv;
  A.st = st;
  A.cfin = ab.cfin;
  A.bar_spins = ab.bar_spins > 0 ? ab.bar_spins : (1ll << 25);
  A.bar_skip = ab.bar_skip;
  A.vc = vc ? *vc : VarCoef{};
  A.jtab = ab.jtab;
  // the largest levels of the mixed path update in a kernel of their own (cooperative launch)
  A.split_update = (dim == 2 && jac_f32 && cluster_size == 0 && !A.vc.a64 && ab.cfin && gk.nodes >= (1ll << 21) &&
                    (int)ipow(coarse_cells + 1, dim) < 128) ? 1 : 0;
  // the barrier words and the abort flag are cleared once per solve (or component call) with
  // the statistics; a completed barrier leaves its count at zero and generations only grow, so
  // the launches of one solve need no reset between them
  cudaError_t e = cudaSuccess;
  if (cluster_size > 0) {
    if (A.vc.a64) return cudaErrorInvalidValue;   // batches and the server take A = I only
    A.bpc = 1;
    cudaLaunchConfig_t cc = {};
    cc.gridDim = dim3(cluster_size);
    cc.blockDim = dim3(nt);
    cc.dynamicSmemBytes = smem;
    cc.stream = s;
    cudaLaunchAttribute ca[1];
    ca[0].id = cudaLaunchAttributeClusterDimension;
    ca[0].val.clusterDim.x = cluster_size;
    ca[0].val.clusterDim.y = 1;
    ca[0].val.clusterDim.z = 1;
    cc.attrs = ca;
    cc.numAttrs = 1;
    if (dim == 2) {
      if (jac_f32) return cudaLaunchKernelEx(&cc, k_augmented_cluster<2, true>, A);
      return cudaLaunchKernelEx(&cc, k_augmented_cluster<2, false>, A);
    }
    if (jac_f32) return cudaLaunchKernelEx(&cc, k_augmented_cluster<3, true>, A);
    return cudaLaunchKernelEx(&cc, k_augmented_cluster<3, false>, A);
  }
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
  const bool v = A.vc.a64 != nullptr;
  if (dim == 2) {
    if (jac_f32)
      e = v ? cudaLaunchKernelEx(&cfg, k_augmented<2, true, true>, A) : cudaLaunchKernelEx(&cfg, k_augmented<2, true, false>, A);
    else
      e = v ? cudaLaunchKernelEx(&cfg, k_augmented<2, false, true>, A)
            : cudaLaunchKernelEx(&cfg, k_augmented<2, false, false>, A);
  } else {
    if (jac_f32)
      e = v ? cudaLaunchKernelEx(&cfg, k_augmented<3, true, true>, A) : cudaLaunchKernelEx(&cfg, k_augmented<3, true, false>, A);
    else
      e = v ? cudaLaunchKernelEx(&cfg, k_augmented<3, false, true>, A)
            : cudaLaunchKernelEx(&cfg, k_augmented<3, false, false>, A);
  }
  if (e != cudaSuccess || !A.split_update) return e;
  int ls = 0;
  while ((1 << ls) < sfine) ++ls;
  // about eight blocks of rows per SM, every block staging the coarse values once
  const unsigned gx = (unsigned)((gk.n + 1 + 255) / 256);
  const long long rows = dim == 2 ? (long long)(gk.n - 1) : (long long)(gk.n - 1) * (gk.n - 1);
  long long gy = (8ll * (ab.sms > 0 ? ab.sms : 152) + gx - 1) / gx;
  if (gy > rows) gy = rows;
  if (gy > 65535) gy = 65535;
  const float* cf = reinterpret_cast<const float*>(ab.cfin);
  if (dim == 2)
    launch_k(k_aug_update<2>, dim3(gx, (unsigned)gy), 256, 0, s, u, gk.n, ls, coarse_cells, cf, out_f64);
  else
    launch_k(k_aug_update<3>, dim3(gx, (unsigned)gy), 256, 0, s, u, gk.n, ls, coarse_cells, cf, out_f64);
  return cudaGetLastError();
}


// The level-1 Newton kernel and the cluster form of the augmented Newton kernel (2D), for
// phase-batched launches.
void phase_kernels_newton(std::vector<PhaseKernel>& out) {
  out.push_back(phase_kernel<&k_level1_newton_body<float>, 256, 2>(&k_level1_newton<float>));
  out.push_back(phase_kernel<&k_level1_newton_body<double>, 256, 2>(&k_level1_newton<double>));
  out.push_back(phase_kernel<&k_augmented_cluster_body<2, true>, Aug<2, true>::NT, 512 / Aug<2, true>::NT>(
      &k_augmented_cluster<2, true>));
  out.push_back(phase_kernel<&k_augmented_cluster_body<2, false>, Aug<2, false>::NT, 512 / Aug<2, false>::NT>(
      &k_augmented_cluster<2, false>));
}

}  // namespace fmg

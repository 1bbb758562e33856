// Mixed-precision path with float-float level data (Algorithm 3.1 step 1 and the FMG
// interpolation of Algorithm 3.2): the level iterate u, the linear right-hand side b of eq.
// (3.4) and g are stored as float-float pairs in the 8-byte slots of the FP64 arrays, and
// the kernels that would otherwise do FP64 arithmetic per node (residual, update, right-hand
// side, interpolation) do it in FP32 error-free transformations instead, so they run at the
// HBM rate.  The FP32 multigrid cycle between residual and update is unchanged.
#include "fmg_ff.cuh"
#include "fmg_internal.cuh"
#include "fmg_phase.cuh"

namespace fmg {

namespace {

constexpr int kB = 128;

unsigned cdiv_u(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// r = b - sigma (2d u - sum of axis neighbours) = b + sigma * neighbour_sum on the interior,
// 0 on the boundary; r32 = fl32(r), and with d32 the first Chebyshev step from zero,
// e = d = e0 r32.
template <int D>
__device__ __forceinline__ void k_residual_ff_body(const double* __restrict__ u, const double* __restrict__ b, int n, ff sigma,
                              float* __restrict__ r32, float* __restrict__ e32, float* __restrict__ d32, float e0,
                              VarCoef vc, int ls) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, l = D == 3 ? blockIdx.z : 0;
  if (i > n) return;
  const long long np = n + 1, pl = np * np;
  const long long c = ((long long)l * np + j) * np + i;
  float v = 0.f;
  if (i > 0 && i < n && j > 0 && j < n && (D == 2 || (l > 0 && l < n))) {
    ff S;
    if (vc.a64) {
      const long long o[3] = {1, np, pl};
      ff nb[2 * D];
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        nb[2 * ax] = ff_load(u + c - o[ax]);
        nb[2 * ax + 1] = ff_load(u + c + o[ax]);
      }
      S = weighted_neighbour_sum_ff<D>(ff_load(u + c), nb, vc, ls, i, j, l);
    } else {
      S = neighbour_sum_ff<D>(u, c, np, pl);
    }
    if (D == 3) S = ff_mul(S, sigma);
    const ff r = ff_add(ff_load(b + c), S);
    v = r.hi + r.lo;
  }
  r32[c] = v;
  const float e = d32 ? e0 * v : 0.f;
  e32[c] = e;
  if (d32) d32[c] = e;
}

// The 3D constant-coefficient residual, a thread walking a strip of kResStrip nodes along z with
// u at z - 1, z, z + 1 in registers (the in-plane neighbours from memory): the same sum of the
// same operands as k_residual_ff<3>, so the same bits, with one plane of u per node from the
// strip instead of three.
constexpr int kResStrip = 8;

__device__ __forceinline__ void k_residual_ff3s_body(const double* __restrict__ u, const double* __restrict__ b, int n,
                                                     ff sigma, float* __restrict__ r32, float* __restrict__ e32,
                                                     float* __restrict__ d32, float e0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const int l0 = blockIdx.z * kResStrip;
  if (i > n) return;
  const long long np = n + 1, pl = np * np;
  long long c = ((long long)l0 * np + j) * np + i;
  const bool inplane = i > 0 && i < n && j > 0 && j < n;
  ff zm = (l0 > 0 && inplane) ? ff_load(u + c - pl) : ff{0.f, 0.f};
  ff zc = inplane ? ff_load(u + c) : ff{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kResStrip; ++k) {
    const int l = l0 + k;
    if (l > n) break;
    const ff zp = (inplane && l + 1 <= n) ? ff_load(u + c + pl) : ff{0.f, 0.f};
    float v = 0.f;
    if (inplane && l > 0 && l < n) {
      const ff um[3] = {ff_load(u + c - 1), ff_load(u + c - np), zm};
      const ff up[3] = {ff_load(u + c + 1), ff_load(u + c + np), zp};
      ff S = neighbour_sum_ff_v<3>(zc, um, up);
      S = ff_mul(S, sigma);
      const ff r = ff_add(ff_load(b + c), S);
      v = r.hi + r.lo;
    }
    r32[c] = v;
    const float e = d32 ? e0 * v : 0.f;
    e32[c] = e;
    if (d32) d32[c] = e;
    zm = zc;
    zc = zp;
    c += pl;
  }
}

__global__ void k_residual_ff3s(const double* __restrict__ u, const double* __restrict__ b, int n, ff sigma,
                                float* __restrict__ r32, float* __restrict__ e32, float* __restrict__ d32, float e0) {
  pdl_start();
  k_residual_ff3s_body(u, b, n, sigma, r32, e32, d32, e0);
}

template <int D>
__global__ void k_residual_ff(const double* __restrict__ u, const double* __restrict__ b, int n, ff sigma,
                              float* __restrict__ r32, float* __restrict__ e32, float* __restrict__ d32, float e0,
                              VarCoef vc, int ls) { pdl_start(); k_residual_ff_body<D>(u, b, n, sigma, r32, e32, d32, e0, vc, ls); }

// b = w (g - a f(u)) on the interior nodes, 0 on the boundary (eq. 3.4 with the vertex rule).
__device__ __forceinline__ void k_nonlinear_rhs_ff_body(const double* __restrict__ u, const double* __restrict__ g, double* __restrict__ b,
                                   int n, int dim, int kind, ff a, double a64, ff w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, l = dim == 3 ? (int)blockIdx.z : 0;
  if (i > n) return;
  const long long np = n + 1;
  const long long idx = ((long long)l * np + j) * np + i;
  ff v{0.f, 0.f};
  if (i > 0 && i < n && j > 0 && j < n && (dim == 2 || (l > 0 && l < n)))
    v = ff_mul(ff_sub(ff_load(g + idx), f_ff(kind, a, a64, ff_load(u + idx))), w);
  ff_store(b + idx, v);
}

__global__ void k_nonlinear_rhs_ff(const double* __restrict__ u, const double* __restrict__ g, double* __restrict__ b,
                                   int n, int dim, int kind, ff a, double a64, ff w) { pdl_start(); k_nonlinear_rhs_ff_body(u, g, b, n, dim, kind, a, a64, w); }

// FMG interpolation u_f = P u_c (the natural inclusion, eq. 3.3) on the interior fine nodes.
template <int D>
__global__ void k_prolong_ff(const double* __restrict__ uc, int nc, double* __restrict__ uf, int nf) {
  pdl_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  const int l = D == 3 ? blockIdx.z + 1 : 0;
  if (i > nf - 1) return;
  const long long cp = nc + 1;
  long long a, z, f;
  if (D == 2) {
    a = (long long)(j >> 1) * cp + (i >> 1);
    z = (long long)((j + 1) >> 1) * cp + ((i + 1) >> 1);
    f = (long long)j * (nf + 1) + i;
  } else {
    a = ((long long)(l >> 1) * cp + (j >> 1)) * cp + (i >> 1);
    z = ((long long)((l + 1) >> 1) * cp + ((j + 1) >> 1)) * cp + ((i + 1) >> 1);
    const long long fp = nf + 1;
    f = ((long long)l * fp + j) * fp + i;
  }
  const ff s = ff_add(ff_load(uc + a), ff_load(uc + z));
  ff_store(uf + f, ff{0.5f * s.hi, 0.5f * s.lo});
}

// The start of a level of Algorithm 3.2 in one pass: the FMG interpolation u = P u_c, the
// right-hand side b = w (g - a f(u)) of eq. (3.4) and the first residual r = b - A_k u of the
// defect correction (with d32: the first Chebyshev step from zero, e = d = e0 r).  The
// interpolated values at the stencil neighbours are formed on the fly from u_c, with the
// same operations as the stored ones, so the result is that of the three separate passes.
template <int D>
__device__ __forceinline__ ff interp_ff(const double* __restrict__ uc, long long cp, int i, int j, int l) {
  long long a, z;
  if (D == 2) {
    a = (long long)(j >> 1) * cp + (i >> 1);
    z = (long long)((j + 1) >> 1) * cp + ((i + 1) >> 1);
  } else {
    a = ((long long)(l >> 1) * cp + (j >> 1)) * cp + (i >> 1);
    z = ((long long)((l + 1) >> 1) * cp + ((j + 1) >> 1)) * cp + ((i + 1) >> 1);
  }
  const ff s = ff_add(ff_load(uc + a), ff_load(uc + z));
  return ff{0.5f * s.hi, 0.5f * s.lo};
}

template <int D>
__global__ void k_level_start_ff(const double* __restrict__ uc, double* __restrict__ u, const double* __restrict__ g,
                                 double* __restrict__ b, int n, int kind, ff a, double a64, ff w, ff sigma,
                                 float* __restrict__ r32, float* __restrict__ e32, float* __restrict__ d32,
                                 float e0, VarCoef vc, int ls) {
  pdl_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, l = D == 3 ? blockIdx.z : 0;
  if (i > n) return;
  const long long np = n + 1;
  const long long cp = (n >> 1) + 1;
  const long long c = ((long long)l * np + j) * np + i;
  auto inner = [&](int x, int y, int z) {
    return x > 0 && x < n && y > 0 && y < n && (D == 2 || (z > 0 && z < n));
  };
  float v = 0.f;
  ff bv{0.f, 0.f};
  if (inner(i, j, l)) {
    const ff U = interp_ff<D>(uc, cp, i, j, l);
    ff_store(u + c, U);
    bv = ff_mul(ff_sub(ff_load(g + c), f_ff(kind, a, a64, U)), w);
    // sum_k (u_k - u_c) as in neighbour_sum_ff, from the interpolated neighbours (zero on the
    // boundary)
    ff nbv[2 * D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      const int dx = ax == 0, dy = ax == 1, dz = ax == 2;
      nbv[2 * ax] = inner(i - dx, j - dy, l - dz) ? interp_ff<D>(uc, cp, i - dx, j - dy, l - dz) : ff{0.f, 0.f};
      nbv[2 * ax + 1] = inner(i + dx, j + dy, l + dz) ? interp_ff<D>(uc, cp, i + dx, j + dy, l + dz) : ff{0.f, 0.f};
    }
    ff S;
    if (vc.a64) {
      S = weighted_neighbour_sum_ff<D>(U, nbv, vc, ls, i, j, l);
    } else {
      float s = 0.f, lo = 0.f;
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        const ff um = nbv[2 * ax], up = nbv[2 * ax + 1];
        float dm, em, dp, ep, t, et;
        two_sum(um.hi, -U.hi, dm, em);
        two_sum(up.hi, -U.hi, dp, ep);
        two_sum(dm, dp, t, et);
        float s2, e2;
        two_sum(s, t, s2, e2);
        s = s2;
        lo += ((em + ep) + (et + e2)) + ((um.lo - U.lo) + (up.lo - U.lo));
      }
      two_sum(s, lo, S.hi, S.lo);
    }
    if (D == 3) S = ff_mul(S, sigma);
    const ff r = ff_add(bv, S);
    v = r.hi + r.lo;
  }
  ff_store(b + c, bv);
  r32[c] = v;
  const float e = d32 ? e0 * v : 0.f;
  e32[c] = e;
  if (d32) d32[c] = e;
}

// The same level start in 2D with each thread walking a strip of rows of one column (lanes
// along x): the interpolated iterate is formed once per node, the rows above and below are
// carried along the strip and the x-neighbours come from the adjacent lanes (every lane forms
// one more value, the one beyond the warp's edge on its side, which lanes 0 and 31 use).  The operations on each node are those of k_level_start_ff, in
// the same order.  Lanes past the last column store nothing.
__device__ __forceinline__ void k_level_start_ff2_body(const double* __restrict__ uc, double* __restrict__ u, const double* __restrict__ g,
                                  double* __restrict__ b, int n, int kind, ff a, double a64, ff w,
                                  float* __restrict__ r32, float* __restrict__ e32, float* __restrict__ d32, float e0,
                                  int strip, VarCoef vc, int ls) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool act = i <= n;
  const int ic = act ? i : n;
  const int j0 = blockIdx.y * strip;
  const long long np = n + 1;
  const long long cp = (n >> 1) + 1;
  auto inner = [&](int x, int y) { return x > 0 && x < n && y > 0 && y < n; };
  auto U = [&](int x, int y) { return inner(x, y) ? interp_ff<2>(uc, cp, x, y, 0) : ff{0.f, 0.f}; };
  ff um = U(ic, j0 - 1), ucur = U(ic, j0);
  for (int r = 0; r < strip; ++r) {
    const int j = j0 + r;
    if (j > n) break;
    const ff up = U(ic, j + 1);
    // the edge value without a branch: lane 0 needs x - 1, lane 31 x + 1
    const ff ve = U(lane == 0 ? ic - 1 : (act ? ic + 1 : n), j);
    const ff sl{__shfl_up_sync(0xffffffffu, ucur.hi, 1), __shfl_up_sync(0xffffffffu, ucur.lo, 1)};
    const ff sr{__shfl_down_sync(0xffffffffu, ucur.hi, 1), __shfl_down_sync(0xffffffffu, ucur.lo, 1)};
    const ff left = lane == 0 ? ve : sl;
    const ff right = lane == 31 ? ve : sr;
    const long long c = (long long)j * np + ic;
    float v = 0.f;
    ff bv{0.f, 0.f};
    if (act && inner(ic, j)) {
      const ff Uc = ucur;
      ff_store(u + c, Uc);
      bv = ff_mul(ff_sub(ff_load(g + c), f_ff(kind, a, a64, Uc)), w);
      ff S;
      if (vc.a64) {
        const ff nb[4] = {left, right, um, up};
        S = weighted_neighbour_sum_ff<2>(Uc, nb, vc, ls, ic, j, 0);
      } else {
        float s = 0.f, lo = 0.f;
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
          const ff nm = ax == 0 ? left : um;
          const ff nq = ax == 0 ? right : up;
          float dm, em, dp, ep, t, et;
          two_sum(nm.hi, -Uc.hi, dm, em);
          two_sum(nq.hi, -Uc.hi, dp, ep);
          two_sum(dm, dp, t, et);
          float s2, e2;
          two_sum(s, t, s2, e2);
          s = s2;
          lo += ((em + ep) + (et + e2)) + ((nm.lo - Uc.lo) + (nq.lo - Uc.lo));
        }
        two_sum(s, lo, S.hi, S.lo);
      }
      const ff rr = ff_add(bv, S);
      v = rr.hi + rr.lo;
    }
    if (act) {
      ff_store(b + c, bv);
      r32[c] = v;
      const float e = d32 ? e0 * v : 0.f;
      e32[c] = e;
      if (d32) d32[c] = e;
    }
    um = ucur;
    ucur = up;
  }
}

__global__ void k_level_start_ff2(const double* __restrict__ uc, double* __restrict__ u, const double* __restrict__ g,
                                  double* __restrict__ b, int n, int kind, ff a, double a64, ff w,
                                  float* __restrict__ r32, float* __restrict__ e32, float* __restrict__ d32, float e0,
                                  int strip, VarCoef vc, int ls) { pdl_start(); k_level_start_ff2_body(uc, u, g, b, n, kind, a, a64, w, r32, e32, d32, e0, strip, vc, ls); }

__device__ __forceinline__ void k_add_f32_ff_body(double* __restrict__ uff, const float* __restrict__ e, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ff_store(uff + i, ff_add_f(ff_load(uff + i), e[i]));
}

__global__ void k_add_f32_ff(double* __restrict__ uff, const float* __restrict__ e, long long n) { pdl_start(); k_add_f32_ff_body(uff, e, n); }

__global__ void k_ff_from_f64(const double* __restrict__ s, double* __restrict__ d, long long n) {
  pdl_start();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ff_store(d + i, ff_from_double(s[i]));
}

__global__ void k_ff_to_f64(const double* __restrict__ s, double* __restrict__ d, long long n) {
  pdl_start();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = ff_to_double_fast(ff_load(s + i));
}

}  // namespace

// ============================================================================ launchers

// fine cells per coarse cell of a level with n cells per side, as a power of two (VarCoef)
int vc_level_shift(const VarCoef* vc, int n) {
  int ls = 0;
  while (vc && vc->a64 && (vc->nc << ls) < n) ++ls;
  return ls;
}

cudaError_t launch_residual_ff(int dim, LevelGeo g, const double* u_ff, const double* b_ff, float* r32, float* e32,
                               cudaStream_t s, float* d32, double e0, const VarCoef* vc) {
  const int n = g.n;
  const dim3 grid(cdiv_u(n + 1, kB), n + 1, dim == 3 ? n + 1 : 1);
  const VarCoef v = vc ? *vc : VarCoef{};
  const int ls = vc_level_shift(vc, n);
  if (dim == 2)
    launch_k(k_residual_ff<2>, grid, kB, 0, s, u_ff, b_ff, n, ff{1.f, 0.f}, r32, e32, d32, (float)e0, v, ls);
  else if (v.a64)
    launch_k(k_residual_ff<3>, grid, kB, 0, s, u_ff, b_ff, n, ff_from_double(1.0 / n), r32, e32, d32, (float)e0, v, ls);
  else
    launch_k(k_residual_ff3s, dim3(grid.x, n + 1, cdiv_u(n + 1, kResStrip)), kB, 0, s, u_ff, b_ff, n, ff_from_double(1.0 / n),
                                                                               r32, e32, d32, (float)e0);
  return cudaGetLastError();
}

cudaError_t launch_nonlinear_rhs_ff(int dim, LevelGeo g, const double* u_ff, const double* g_ff, double* b_ff,
                                    int kind, double a, cudaStream_t s) {
  const double h = 1.0 / g.n;
  const double w = dim == 2 ? h * h : h * h * h;
  const dim3 grid(cdiv_u(g.n + 1, kB), g.n + 1, dim == 3 ? g.n + 1 : 1);
  launch_k(k_nonlinear_rhs_ff, grid, kB, 0, s, u_ff, g_ff, b_ff, g.n, dim, kind, ff_from_double(a), a, ff_from_double(w));
  return cudaGetLastError();
}

cudaError_t launch_prolong_ff(int dim, LevelGeo gc, const double* uc_ff, LevelGeo gf, double* uf_ff, cudaStream_t s) {
  const int nf = gf.n;
  const dim3 grid(cdiv_u(nf - 1, kB), nf - 1, dim == 3 ? nf - 1 : 1);
  if (dim == 2)
    launch_k(k_prolong_ff<2>, grid, kB, 0, s, uc_ff, gc.n, uf_ff, nf);
  else
    launch_k(k_prolong_ff<3>, grid, kB, 0, s, uc_ff, gc.n, uf_ff, nf);
  return cudaGetLastError();
}

cudaError_t launch_level_start_ff(int dim, LevelGeo gc, const double* uc_ff, LevelGeo g, double* u_ff,
                                  const double* g_ff, double* b_ff, int kind, double a, float* r32, float* e32,
                                  float* d32, double e0, cudaStream_t s, const VarCoef* vc) {
  const int n = g.n;
  if (gc.n * 2 != n) return cudaErrorInvalidValue;
  const VarCoef v = vc ? *vc : VarCoef{};
  const int ls = vc_level_shift(vc, n);
  const double h = 1.0 / n;
  const double w = dim == 2 ? h * h : h * h * h;
  const dim3 grid(cdiv_u(n + 1, kB), n + 1, dim == 3 ? n + 1 : 1);
  if (dim == 2) {
    // strips of up to 8 rows, shorter on small levels so that the grid keeps ~1000 blocks
    int strip = 8;
    while (strip > 1 && (long long)cdiv_u(n + 1, kB) * cdiv_u(n + 1, strip) < 1024) strip >>= 1;
    launch_k(k_level_start_ff2, dim3(cdiv_u(n + 1, kB), cdiv_u(n + 1, strip)), kB, 0, s, 
        uc_ff, u_ff, g_ff, b_ff, n, kind, ff_from_double(a), a, ff_from_double(w), r32, e32, d32, (float)e0, strip, v,
        ls);
  } else
    launch_k(k_level_start_ff<3>, grid, kB, 0, s, uc_ff, u_ff, g_ff, b_ff, n, kind, ff_from_double(a), a, ff_from_double(w),
                                            ff_from_double(h), r32, e32, d32, (float)e0, v, ls);
  return cudaGetLastError();
}

cudaError_t launch_add_f32_ff(LevelGeo g, double* u_ff, const float* e32, cudaStream_t s) {
  launch_k(k_add_f32_ff, cdiv_u(g.nodes, 256), 256, 0, s, u_ff, e32, g.nodes);
  return cudaGetLastError();
}

namespace {

// The right-hand side of every level from the fine g just copied in, in one launch: the fine
// g's boundary ring set to zero in place; each coarser level's g the fine values at its nodes (the
// nodal injection of the nested hierarchy: node (i, j[, l]) of level k is fine node
// (i, j[, l]) n_L / n_k), zero on its boundary; and with ff the float-float copy of every level.
// Blocks boff[k] .. boff[k+1]-1 take level k.  The fine level's blocks write only its boundary
// ring and the coarser levels' blocks read only fine interior nodes, so they do not race.
struct RhsLevels {
  double* g[kMaxLevels];
  double* gf[kMaxLevels];
  int n[kMaxLevels];
  long long nodes[kMaxLevels];
  long long boff[kMaxLevels + 1];
  int nlev, dim, ff;
};

__global__ void k_rhs_levels(const __grid_constant__ RhsLevels R) {
  pdl_start();
  const long long bid = blockIdx.x;
  int k = 0;
  while (k + 1 < R.nlev && bid >= R.boff[k + 1]) ++k;
  const long long idx = (bid - R.boff[k]) * blockDim.x + threadIdx.x;
  if (idx >= R.nodes[k]) return;
  const int top = R.nlev - 1;
  const int n = R.n[k];
  const long long cp = n + 1;
  const int i = (int)(idx % cp), j = (int)((idx / cp) % cp), l = R.dim == 3 ? (int)(idx / (cp * cp)) : 0;
  const bool bnd = i == 0 || i == n || j == 0 || j == n || (R.dim == 3 && (l == 0 || l == n));
  double v;
  if (k == top) {
    v = bnd ? 0.0 : R.g[top][idx];
    if (bnd) R.g[top][idx] = 0.0;
  } else {
    const long long st = R.n[top] / n, fp = R.n[top] + 1;
    v = bnd ? 0.0 : R.g[top][((l * st) * fp + j * st) * fp + i * st];
    R.g[k][idx] = v;
  }
  if (R.ff) ff_store(R.gf[k] + idx, ff_from_double(v));
}

}  // namespace

cudaError_t launch_rhs_levels(int dim, int nlev, const LevelGeo* geo, double* const* g, double* const* gf, bool ff,
                              cudaStream_t s) {
  if (nlev < 1 || nlev > kMaxLevels) return cudaErrorInvalidValue;
  RhsLevels R = {};
  long long off = 0;
  for (int k = 0; k < nlev; ++k) {
    R.g[k] = g[k];
    R.gf[k] = ff ? gf[k] : nullptr;
    R.n[k] = geo[k].n;
    R.nodes[k] = geo[k].nodes;
    R.boff[k] = off;
    off += (geo[k].nodes + 255) / 256;
  }
  R.boff[nlev] = off;
  R.nlev = nlev;
  R.dim = dim;
  R.ff = ff ? 1 : 0;
  if (off < 1 || off > 0x7fffffffll) return cudaErrorInvalidValue;
  launch_k(k_rhs_levels, dim3((unsigned)off), 256, 0, s, R);
  return cudaGetLastError();
}

cudaError_t launch_ff_from_f64(const double* src, double* dst_ff, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  launch_k(k_ff_from_f64, cdiv_u(n, 256), 256, 0, s, src, dst_ff, n);
  return cudaGetLastError();
}

cudaError_t launch_ff_to_f64(const double* src_ff, double* dst, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  launch_k(k_ff_to_f64, cdiv_u(n, 256), 256, 0, s, src_ff, dst, n);
  return cudaGetLastError();
}


// The 2D float-float kernels of the mixed solve, for phase-batched launches.
void phase_kernels_ff(std::vector<PhaseKernel>& out) {
  out.push_back(phase_kernel<&k_residual_ff_body<2>, kB, 16>(&k_residual_ff<2>));
  out.push_back(phase_kernel<&k_nonlinear_rhs_ff_body, kB, 1>(&k_nonlinear_rhs_ff));
  out.push_back(phase_kernel<&k_level_start_ff2_body, kB, 9>(&k_level_start_ff2));
  out.push_back(phase_kernel<&k_add_f32_ff_body, 256, 1>(&k_add_f32_ff));
}

}  // namespace fmg

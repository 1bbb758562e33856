// Matrix-free stencil kernels of the multigrid cycle (Algorithm 3.1 step 1, eq. 3.4-3.5)
// and the pointwise steps of the full multigrid schedule (Algorithm 3.2).
//
// Operators (P1 elements on the nested right-triangle / Kuhn meshes of Sec. 3):
//   A_k     = sigma_k * (2d-point Laplacian),   sigma_k = h_k^(d-2)
//   P_k     = nodal interpolation V_{h_{k-1}} -> V_{h_k}: a fine node at the midpoint of a
//             coarse edge takes the mean of the edge's two end values; every edge of these
//             meshes joins a coarse node z to z + e with e a nonzero 0/1 vector, so the two
//             ends of the edge through fine node x are floor(x/2) and ceil(x/2)
//   P_k^T   = restriction: coarse node z gathers 1 x r(2z) + 1/2 x r(2z +- e) over the
//             2^d - 1 edge directions e
// Red-black Gauss-Seidel: red nodes have i+j[+l] even.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "fmg_ff.cuh"
#include "fmg_internal.cuh"
#include "fmg_phase.cuh"

namespace fmg {

namespace {

constexpr int kBlock = 128;
constexpr int kMaxCoarseN = 64;   // level-1 unknowns (2D: (1/H - 1)^2 <= 49, 3D: <= 27)

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------------ red-black Gauss-Seidel
template <typename T>
__device__ __forceinline__ void k_rbgs2_body(T* __restrict__ u, const T* __restrict__ b, int n, int colour) {
  const int j = blockIdx.y + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int par = (colour + j) & 1;
  const int i = par ? 2 * t + 1 : 2 * t + 2;
  if (i > n - 1) return;
  const long long np = n + 1;
  const long long c = (long long)j * np + i;
  const T s = (u[c - 1] + u[c + 1]) + (u[c - np] + u[c + np]);
  u[c] = (b[c] + s) * T(0.25);
}

template <typename T>
__global__ void k_rbgs2(T* __restrict__ u, const T* __restrict__ b, int n, int colour) { pdl_start(); k_rbgs2_body<T>(u, b, n, colour); }

template <typename T>
__global__ void k_rbgs3(T* __restrict__ u, const T* __restrict__ b, int n, int colour, T bscale, T inv6) {
  pdl_start();
  const int j = blockIdx.y + 1;
  const int l = blockIdx.z + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int par = (colour + j + l) & 1;
  const int i = par ? 2 * t + 1 : 2 * t + 2;
  if (i > n - 1) return;
  const long long np = n + 1;
  const long long pl = np * np;
  const long long c = ((long long)l * np + j) * np + i;
  const T s = ((u[c - 1] + u[c + 1]) + (u[c - np] + u[c + np])) + (u[c - pl] + u[c + pl]);
  u[c] = (b[c] * bscale + s) * inv6;
}

// ------------------------------------------------------------------ Chebyshev-Jacobi step
// z = D^{-1}(b - A u) = (b / sigma + sum of the 2d neighbours) / 2d - u; d <- cd d + cr z;
// uo = u + d.  Every interior node at once (colour-free): u is read, uo written.  A thread
// walks a strip of `strip` (<= kChebStrip) nodes along the outermost axis (y in 2D, z in 3D),
// keeping the previous, current and next values of u on that axis in registers, so u is read
// once per node from memory along the strip plus the in-plane neighbours from cache.
constexpr int kChebStrip = 8;

// With ec (the first post-smoothing step of a cycle) the iterate is u + P e_c: the coarse
// correction prolongated on the fly (two coarse values per fine node, P of eq. 3.3) for the
// node and its stencil neighbours, in place of a separate prolongation pass.
template <typename T, int D>
__device__ __forceinline__ T prolong_at(const T* __restrict__ ec, long long cp, int i, int j, int l) {
  if (D == 2)
    return T(0.5) * (ec[(long long)(j >> 1) * cp + (i >> 1)] + ec[(long long)((j + 1) >> 1) * cp + ((i + 1) >> 1)]);
  return T(0.5) * (ec[((long long)(l >> 1) * cp + (j >> 1)) * cp + (i >> 1)] +
                   ec[((long long)((l + 1) >> 1) * cp + ((j + 1) >> 1)) * cp + ((i + 1) >> 1)]);
}

template <typename T, int D, bool PROL>
__device__ __forceinline__ void k_cheb_body(const T* __restrict__ u, T* __restrict__ uo, T* __restrict__ d, const T* __restrict__ b, int n,
                       T bscale, T cd, T cr, int first, int strip, const T* __restrict__ ec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = D == 3 ? blockIdx.y + 1 : 0;                 // in-plane row (3D only)
  const int z0 = (D == 2 ? blockIdx.y : blockIdx.z) * strip + 1;   // strip start (outer axis)
  if (i > n - 1) return;
  const long long np = n + 1;
  const long long so = D == 2 ? np : np * np;                // stride of the outer axis
  const long long cp = (n >> 1) + 1;                         // coarse row length (PROL)
  // iterate at fine node (x, y[, w]) with the outer axis last: u (+ P e_c)
  auto iter = [&](long long cc, int x, int y, int w) -> T {
    T v = u[cc];
    if (PROL) v += D == 2 ? prolong_at<T, 2>(ec, cp, x, y, 0) : prolong_at<T, 3>(ec, cp, x, y, w);
    return v;
  };
  long long c = (D == 2 ? (long long)z0 * np : ((long long)z0 * np + j) * np) + i;
  T um = D == 2 ? iter(c - so, i, z0 - 1, 0) : iter(c - so, i, j, z0 - 1);
  T uc = D == 2 ? iter(c, i, z0, 0) : iter(c, i, j, z0);
  const T inv2d = T(1) / T(2 * D);
#pragma unroll
  for (int r = 0; r < kChebStrip; ++r) {
    if (r >= strip || z0 + r > n - 1) break;
    const int z = z0 + r;
    const T up = D == 2 ? iter(c + so, i, z + 1, 0) : iter(c + so, i, j, z + 1);
    T s;
    if (D == 2) {
      s = (iter(c - 1, i - 1, z, 0) + iter(c + 1, i + 1, z, 0)) + (um + up);
    } else {
      s = (iter(c - 1, i - 1, j, z) + iter(c + 1, i + 1, j, z)) + (um + up);
      s += iter(c - np, i, j - 1, z) + iter(c + np, i, j + 1, z);
    }
    const T zr = (b[c] * bscale + s) * inv2d - uc;
    const T dn = first ? cr * zr : cd * d[c] + cr * zr;
    d[c] = dn;
    uo[c] = uc + dn;
    um = uc;
    uc = up;
    c += so;
  }
}

template <typename T, int D, bool PROL>
__global__ void k_cheb(const T* __restrict__ u, T* __restrict__ uo, T* __restrict__ d, const T* __restrict__ b, int n,
                       T bscale, T cd, T cr, int first, int strip, const T* __restrict__ ec) { pdl_start(); k_cheb_body<T, D, PROL>(u, uo, d, b, n, bscale, cd, cr, first, strip, ec); }

// The last Chebyshev step of the mixed path's top-level FP32 cycle fused with its update
// u64 += u + d_new (the new correction is neither stored nor read back); FF: u64 holds
// float-float values (the solve's level data) instead of FP64 ones (the ops' arrays).
template <int D, bool FF>
__device__ __forceinline__ void k_cheb_add64_body(const float* __restrict__ u, const float* __restrict__ d, const float* __restrict__ b,
                             double* __restrict__ u64, int n, float bscale, float cd, float cr, int first, int strip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = D == 3 ? blockIdx.y + 1 : 0;
  const int z0 = (D == 2 ? blockIdx.y : blockIdx.z) * strip + 1;
  if (i > n - 1) return;
  const long long np = n + 1;
  const long long so = D == 2 ? np : np * np;
  long long c = (D == 2 ? (long long)z0 * np : ((long long)z0 * np + j) * np) + i;
  float um = u[c - so], uc = u[c];
  const float inv2d = 1.0f / (2 * D);
#pragma unroll
  for (int r = 0; r < kChebStrip; ++r) {
    if (r >= strip || z0 + r > n - 1) break;
    const float up = u[c + so];
    float s = (u[c - 1] + u[c + 1]) + (um + up);
    if (D == 3) s += u[c - np] + u[c + np];
    const float zr = (b[c] * bscale + s) * inv2d - uc;
    const float dn = first ? cr * zr : cd * d[c] + cr * zr;
    if (FF)
      ff_store(u64 + c, ff_add_f(ff_load(u64 + c), uc + dn));
    else
      u64[c] += (double)(uc + dn);
    um = uc;
    uc = up;
    c += so;
  }
}

template <int D, bool FF>
__global__ void k_cheb_add64(const float* __restrict__ u, const float* __restrict__ d, const float* __restrict__ b,
                             double* __restrict__ u64, int n, float bscale, float cd, float cr, int first, int strip) { pdl_start(); k_cheb_add64_body<D, FF>(u, d, b, u64, n, bscale, cd, cr, first, strip); }

template <typename T>
__device__ __forceinline__ void k_copy_t_body(const T* __restrict__ s, T* __restrict__ d, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = s[i];
}

template <typename T>
__global__ void k_copy_t(const T* __restrict__ s, T* __restrict__ d, long long n) { pdl_start(); k_copy_t_body<T>(s, d, n); }

__global__ void k_to_f32(const double* __restrict__ s, float* __restrict__ d, long long n) {
  pdl_start();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (float)s[i];
}

// ------------------------------------------------------------------ residual + restriction
template <typename T>
__device__ __forceinline__ T res2(const T* __restrict__ u, const T* __restrict__ b, long long c, long long np) {
  return b[c] - (T(4) * u[c] - ((u[c - 1] + u[c + 1]) + (u[c - np] + u[c + np])));
}

template <typename T>
__device__ __forceinline__ T res3(const T* __restrict__ u, const T* __restrict__ b, long long c, long long np,
                                  long long pl, T sigma) {
  return b[c] - sigma * (T(6) * u[c] - (((u[c - 1] + u[c + 1]) + (u[c - np] + u[c + np])) + (u[c - pl] + u[c + pl])));
}

// With dc != NULL the coarse level's first Chebyshev step from its zero start is taken here
// too: u_c = d_c = e0 b_c (e0 = cr_0 / diag of the coarse level).
// 2D: a thread per coarse column I walks a strip of coarse rows.  Per fine row it loads u at the
// five fine columns 2I-2 .. 2I+2 (neighbouring threads' loads overlap in L1) and forms the
// residuals at 2I-1, 2I, 2I+1; the previous fine row's residuals and the rows of u stay in
// registers.  So a thread reads each fine row of u once and forms three residuals per fine row
// instead of seven residuals from 35 loads per coarse node.  The residual and the restriction's sum are the
// per-node kernel's expressions in the same order, so the results are the same.  The strip length S
// is a compile-time constant and its loop unrolled, so that all of a thread's row loads are issued
// together (a strip costs one memory latency); larger levels take longer strips.

template <typename TF>
struct RRow {
  TF ll, l, c, r, rr;   // u at the fine columns 2I-2 .. 2I+2 of one fine row
};

template <typename TF, typename TC, int S>
__device__ __forceinline__ void k_resrestrict2_body(const TF* __restrict__ u, const TF* __restrict__ b, int nf,
                                                    TC* __restrict__ bc, TC* __restrict__ uc, int ncells,
                                                    TC* __restrict__ dc, TC e0) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int J0 = blockIdx.y * S + 1;
  const int J1 = min(J0 + S, ncells);   // coarse rows J0 .. J1-1
  const long long np = nf + 1;
  const int x0 = 2 * I;
  const bool v0 = x0 <= nf, v1 = x0 + 1 <= nf;   // the thread's columns inside the row
  // u at the five columns 2I-2 .. 2I+2 of fine row y (outside the row: 0; those columns are
  // only read by threads whose coarse column is outside the level)
  auto load_row = [&](int y) {
    const long long o = (long long)y * np;
    RRow<TF> w;
    w.ll = x0 - 2 <= nf ? u[o + x0 - 2] : TF(0);
    w.l = x0 - 1 <= nf ? u[o + x0 - 1] : TF(0);
    w.c = v0 ? u[o + x0] : TF(0);
    w.r = v1 ? u[o + x0 + 1] : TF(0);
    w.rr = x0 + 2 <= nf ? u[o + x0 + 2] : TF(0);
    return w;
  };
  // residuals of fine row y at columns 2I-1, 2I, 2I+1 from the rows y-1, y, y+1
  auto res_row = [&](int y, const RRow<TF>& m, const RRow<TF>& c, const RRow<TF>& p, TF& rl, TF& rc, TF& rr) {
    const long long o = (long long)y * np;
    const TF blv = x0 - 1 <= nf ? b[o + x0 - 1] : TF(0);
    const TF bcv = v0 ? b[o + x0] : TF(0);
    const TF brv = v1 ? b[o + x0 + 1] : TF(0);
    rl = blv - (TF(4) * c.l - ((c.ll + c.c) + (m.l + p.l)));
    rc = bcv - (TF(4) * c.c - ((c.l + c.r) + (m.c + p.c)));
    rr = brv - (TF(4) * c.r - ((c.c + c.rr) + (m.r + p.r)));
  };
  if (J0 >= J1) return;   // uniform over the block
  RRow<TF> rm = load_row(2 * J0 - 2), r0 = load_row(2 * J0 - 1), rp = load_row(2 * J0);
  TF pl, pc, pr;   // residuals of fine row 2J - 1
  res_row(2 * J0 - 1, rm, r0, rp, pl, pc, pr);
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const int J = J0 + k;
    if (J >= J1) break;   // uniform over the block
    rm = r0;
    r0 = rp;
    rp = load_row(2 * J + 1);
    TF al, ac, ar;   // fine row 2J
    res_row(2 * J, rm, r0, rp, al, ac, ar);
    rm = r0;
    r0 = rp;
    rp = load_row(2 * J + 2);
    TF ql, qc, qr;   // fine row 2J + 1
    res_row(2 * J + 1, rm, r0, rp, ql, qc, qr);
    if (I <= ncells - 1) {
      // b_c = r(2I, 2J) + (r(2I+1, 2J) + r(2I-1, 2J) + r(2I, 2J+1) + r(2I, 2J-1)
      //       + r(2I+1, 2J+1) + r(2I-1, 2J-1)) / 2
      const TF e = (ar + al) + (qc + pc) + (qr + pl);
      const long long cc = (long long)J * (ncells + 1) + I;
      const TC bv = (TC)(ac + TF(0.5) * e);
      bc[cc] = bv;
      const TC e1 = dc ? e0 * bv : TC(0);
      uc[cc] = e1;
      if (dc) dc[cc] = e1;
    }
    pl = ql;
    pc = qc;
    pr = qr;
  }
  (void)pr;
}

template <typename TF, typename TC, int S>
__global__ void k_resrestrict2(const TF* __restrict__ u, const TF* __restrict__ b, int nf, TC* __restrict__ bc,
                               TC* __restrict__ uc, int ncells, TC* __restrict__ dc, TC e0) {
  pdl_start();
  k_resrestrict2_body<TF, TC, S>(u, b, nf, bc, uc, ncells, dc, e0);
}

// Coarse rows per thread of the 2D residual + restriction: 1 on small levels (parallelism), up
// to 4 on large ones (fewer loads per node).
inline int rr_strip(int ncells) { return ncells <= 128 ? 1 : (ncells <= 512 ? 2 : 4); }

template <typename TF, typename TC>
__global__ void k_resrestrict3(const TF* __restrict__ u, const TF* __restrict__ b, int nf, TF sigma,
                               TC* __restrict__ bc, TC* __restrict__ uc, int ncells, TC* __restrict__ dc, TC e0) {
  pdl_start();
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int J = blockIdx.y + 1;
  const int L = blockIdx.z + 1;
  if (I > ncells - 1) return;
  const long long np = nf + 1;
  const long long pl = np * np;
  const long long F = ((long long)(2 * L) * np + 2 * J) * np + 2 * I;
  const long long o[7] = {1, np, pl, 1 + np, 1 + pl, np + pl, 1 + np + pl};
  TF r = res3(u, b, F, np, pl, sigma);
  TF e = TF(0);
#pragma unroll
  for (int q = 0; q < 7; ++q) e += res3(u, b, F + o[q], np, pl, sigma) + res3(u, b, F - o[q], np, pl, sigma);
  const long long ncp = ncells + 1;
  const long long cc = ((long long)L * ncp + J) * ncp + I;
  const TC bv = (TC)(r + TF(0.5) * e);
  bc[cc] = bv;
  const TC e1 = dc ? e0 * bv : TC(0);
  uc[cc] = e1;
  if (dc) dc[cc] = e1;
}

// ------------------------------------------------------------------ residual on one level
// With d32 != NULL the first Chebyshev step of the FP32 cycle, which starts from a zero
// correction, is taken here too: e = d = e0 r (e0 = cr_0 / diag).
__global__ void k_residual2(const double* __restrict__ u, const double* __restrict__ b, int n,
                            double* __restrict__ r, float* __restrict__ r32, float* __restrict__ e32,
                            float* __restrict__ d32, float e0) {
  pdl_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i > n) return;
  const long long np = n + 1;
  const long long c = (long long)j * np + i;
  double v = 0.0;
  if (i > 0 && i < n && j > 0 && j < n) v = res2(u, b, c, np);
  if (r) r[c] = v;
  if (r32) {
    const float vf = (float)v;
    r32[c] = vf;
    const float e = d32 ? e0 * vf : 0.0f;
    e32[c] = e;
    if (d32) d32[c] = e;
  }
}

__global__ void k_residual3(const double* __restrict__ u, const double* __restrict__ b, int n, double sigma,
                            double* __restrict__ r, float* __restrict__ r32, float* __restrict__ e32,
                            float* __restrict__ d32, float e0) {
  pdl_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const int l = blockIdx.z;
  if (i > n) return;
  const long long np = n + 1;
  const long long pl = np * np;
  const long long c = ((long long)l * np + j) * np + i;
  double v = 0.0;
  if (i > 0 && i < n && j > 0 && j < n && l > 0 && l < n) v = res3(u, b, c, np, pl, sigma);
  if (r) r[c] = v;
  if (r32) {
    const float vf = (float)v;
    r32[c] = vf;
    const float e = d32 ? e0 * vf : 0.0f;
    e32[c] = e;
    if (d32) d32[c] = e;
  }
}

// ------------------------------------------------------------------ variable coefficient
// The stencil kernels for A(x) != I (VarCoef): the weights w_e of the 2d axis edges at each node
// come from the per-cell table (edge_weights_t), A u = s sum_e w_e (u_c - u_e) with s = 1 in 2D
// and h in 3D.  Red-black Gauss-Seidel: u_c = (b / s + sum_e w_e u_e) / sum_e w_e.
template <int D>
__device__ __forceinline__ void vc_offsets(long long np, long long* o) {
  o[0] = -1;
  o[1] = 1;
  o[2] = -np;
  o[3] = np;
  if (D == 3) {
    o[4] = -np * np;
    o[5] = np * np;
  }
}

template <typename T, int D>
__global__ void k_rbgs_vc(T* __restrict__ u, const T* __restrict__ b, int n, int colour, int ls, VarCoef vc) {
  pdl_start();
  const int j = blockIdx.y + 1;
  const int l = D == 3 ? blockIdx.z + 1 : 0;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int par = (colour + j + l) & 1;
  const int i = par ? 2 * t + 1 : 2 * t + 2;
  if (i > n - 1) return;
  const long long np = n + 1;
  const long long c = (D == 2 ? (long long)j * np : ((long long)l * np + j) * np) + i;
  long long o[2 * D];
  vc_offsets<D>(np, o);
  T w[2 * D];
  edge_weights_t<D, T>(vc, ls, i, j, l, w);
  T sw = T(0), su = T(0);
#pragma unroll
  for (int e = 0; e < 2 * D; ++e) {
    sw += w[e];
    su += w[e] * u[c + o[e]];
  }
  u[c] = (b[c] * (D == 2 ? T(1) : T(n)) + su) / sw;
}

// r = b - A u at node c (interior), A with the variable coefficient
template <typename T, int D>
__device__ __forceinline__ T res_vc(const T* __restrict__ u, const T* __restrict__ b, long long c, int i, int j, int l,
                                    int n, int ls, const VarCoef& vc) {
  const long long np = n + 1;
  long long o[2 * D];
  vc_offsets<D>(np, o);
  T w[2 * D];
  edge_weights_t<D, T>(vc, ls, i, j, l, w);
  const T uc = u[c];
  T a = T(0);
#pragma unroll
  for (int e = 0; e < 2 * D; ++e) a += w[e] * (uc - u[c + o[e]]);
  return b[c] - (D == 2 ? T(1) : T(1) / T(n)) * a;
}

// residual + restriction with the variable coefficient: b_c = P^T (b - A u) (coarse nodes of
// the interior), u_c = 0 (or the first Chebyshev step, unused with A(x): red-black only)
template <typename TF, typename TC, int D>
__global__ void k_resrestrict_vc(const TF* __restrict__ u, const TF* __restrict__ b, int nf, int ls, VarCoef vc,
                                 TC* __restrict__ bc, TC* __restrict__ uc, int ncells) {
  pdl_start();
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int J = blockIdx.y + 1;
  const int L = D == 3 ? blockIdx.z + 1 : 0;
  if (I > ncells - 1) return;
  const long long np = nf + 1;
  const int fi = 2 * I, fj = 2 * J, fl = 2 * L;
  const long long F = (D == 2 ? (long long)fj * np : ((long long)fl * np + fj) * np) + fi;
  TF r = res_vc<TF, D>(u, b, F, fi, fj, fl, nf, ls, vc);
  TF e = TF(0);
  // the fine nodes at the mesh-edge neighbours of the coarse node: +-(1,0[,0]), +-(0,1[,0]),
  // +-(1,1[,0]) and in 3D +-(0,0,1), +-(1,0,1), +-(0,1,1), +-(1,1,1)
  constexpr int NQ = D == 2 ? 3 : 7;
  const int dq[7][3] = {{1, 0, 0}, {0, 1, 0}, {1, 1, 0}, {0, 0, 1}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const long long off = dq[q][0] + dq[q][1] * np + (D == 3 ? dq[q][2] * np * np : 0);
    e += res_vc<TF, D>(u, b, F + off, fi + dq[q][0], fj + dq[q][1], fl + dq[q][2], nf, ls, vc) +
         res_vc<TF, D>(u, b, F - off, fi - dq[q][0], fj - dq[q][1], fl - dq[q][2], nf, ls, vc);
  }
  const long long ncp = ncells + 1;
  const long long cc = (D == 2 ? (long long)J * ncp : ((long long)L * ncp + J) * ncp) + I;
  bc[cc] = (TC)(r + TF(0.5) * e);
  uc[cc] = TC(0);
}

// FP64 residual on one level with the variable coefficient (with r32: its FP32 copy, e = 0)
template <int D>
__global__ void k_residual_vc(const double* __restrict__ u, const double* __restrict__ b, int n, int ls, VarCoef vc,
                              double* __restrict__ r, float* __restrict__ r32, float* __restrict__ e32) {
  pdl_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const int l = D == 3 ? blockIdx.z : 0;
  if (i > n) return;
  const long long np = n + 1;
  const long long c = (D == 2 ? (long long)j * np : ((long long)l * np + j) * np) + i;
  double v = 0.0;
  if (i > 0 && i < n && j > 0 && j < n && (D == 2 || (l > 0 && l < n))) v = res_vc<double, D>(u, b, c, i, j, l, n, ls, vc);
  if (r) r[c] = v;
  if (r32) {
    r32[c] = (float)v;
    e32[c] = 0.f;
  }
}

int vc_ls(const VarCoef& vc, int n) {
  int ls = 0;
  while ((vc.nc << ls) < n) ++ls;
  return ls;
}

// ------------------------------------------------------------------ prolongation (+ correction)
template <typename TF, typename TC>
__device__ __forceinline__ void k_prolong2_body(const TC* __restrict__ e, int nc, TF* __restrict__ u, int nf, int add) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > nf - 1) return;
  const long long cp = nc + 1;
  const long long a = (long long)(j >> 1) * cp + (i >> 1);
  const long long z = (long long)((j + 1) >> 1) * cp + ((i + 1) >> 1);
  const TF v = TF(0.5) * ((TF)e[a] + (TF)e[z]);
  const long long f = (long long)j * (nf + 1) + i;
  u[f] = add ? u[f] + v : v;
}

template <typename TF, typename TC>
__global__ void k_prolong2(const TC* __restrict__ e, int nc, TF* __restrict__ u, int nf, int add) { pdl_start(); k_prolong2_body<TF, TC>(e, nc, u, nf, add); }

template <typename TF, typename TC>
__global__ void k_prolong3(const TC* __restrict__ e, int nc, TF* __restrict__ u, int nf, int add) {
  pdl_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  const int l = blockIdx.z + 1;
  if (i > nf - 1) return;
  const long long cp = nc + 1;
  const long long a = ((long long)(l >> 1) * cp + (j >> 1)) * cp + (i >> 1);
  const long long z = ((long long)((l + 1) >> 1) * cp + ((j + 1) >> 1)) * cp + ((i + 1) >> 1);
  const TF v = TF(0.5) * ((TF)e[a] + (TF)e[z]);
  const long long fp = nf + 1;
  const long long f = ((long long)l * fp + j) * fp + i;
  u[f] = add ? u[f] + v : v;
}

// ------------------------------------------------------------------ pointwise kernels
__global__ void k_add_f32(double* __restrict__ u, const float* __restrict__ e, long long n) {
  pdl_start();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] += (double)e[i];
}

// b = w (g - f(u)) on the interior nodes, 0 on the boundary; one thread per node of row
// (j[, l]) = (blockIdx.y[, blockIdx.z]), so no index division.
__device__ __forceinline__ void k_nonlinear_rhs_body(const double* __restrict__ u, const double* __restrict__ g, double* __restrict__ b,
                                int n, int dim, int kind, double a, double w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, l = dim == 3 ? (int)blockIdx.z : 0;
  if (i > n) return;
  const long long np = n + 1;
  const long long idx = ((long long)l * np + j) * np + i;
  const bool inner = i > 0 && i < n && j > 0 && j < n && (dim == 2 || (l > 0 && l < n));
  double v = 0.0;
  if (inner) v = w * (g[idx] - f_only<double>(kind, a, u[idx]));
  b[idx] = v;
}

__global__ void k_nonlinear_rhs(const double* __restrict__ u, const double* __restrict__ g, double* __restrict__ b,
                                int n, int dim, int kind, double a, double w) { pdl_start(); k_nonlinear_rhs_body(u, g, b, n, dim, kind, a, w); }

__global__ void k_copy(const double* __restrict__ s, double* __restrict__ d, long long n) {
  pdl_start();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = s[i];
}

// ------------------------------------------------------------------ coarsest solve (dense inverse)
// Unknown r of level 1 <-> interior node (r % m + 1, (r / m) % m + 1, r / m^2 + 1), m = n1 - 1.
__device__ __forceinline__ long long coarse_node(int r, int m, int dim) {
  const long long np = m + 2;
  const int i = r % m + 1;
  const int j = (r / m) % m + 1;
  if (dim == 2) return (long long)j * np + i;
  const int l = r / (m * m) + 1;
  return ((long long)l * np + j) * np + i;
}

// u = A_1^{-1} b on the level-1 unknowns.  b is staged in shared memory; A_1^{-1} is
// symmetric, so thread r reads column r (coalesced across threads).
template <typename T>
__device__ __forceinline__ void k_coarse_solve_body(const double* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ u, int m,
                               int N, int dim) {
  extern __shared__ double bs[];
  for (int c = threadIdx.x; c < N; c += blockDim.x) bs[c] = (double)b[coarse_node(c, m, dim)];
  __syncthreads();
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    double a0 = 0.0, a1 = 0.0;
    int c = 0;
    for (; c + 1 < N; c += 2) {
      a0 = fma(Ainv[(long long)c * N + r], bs[c], a0);
      a1 = fma(Ainv[(long long)(c + 1) * N + r], bs[c + 1], a1);
    }
    if (c < N) a0 = fma(Ainv[(long long)c * N + r], bs[c], a0);
    u[coarse_node(r, m, dim)] = (T)(a0 + a1);
  }
}

template <typename T>
__global__ void k_coarse_solve(const double* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ u, int m,
                               int N, int dim) { pdl_start(); k_coarse_solve_body<T>(Ainv, b, u, m, N, dim); }

// ------------------------------------------------------------------ coarse V-cycle in one CTA
// The V(nu_pre, nu_post) cycle on levels jtop..1 with every level's u and b in shared
// memory: the same red-black sweeps, restriction P^T, exact level-1 solve (dense
// A_1^{-1} in FP64) and prolongation as the per-level kernels, separated by __syncthreads
// instead of launches.  Level jtop's u and b are read from and u written back to global
// memory.  Level j has n0 << (j-1) cells per side.
template <typename T, int D>
struct CoarseLevel {
  int n;        // cells per side (a power of two)
  int lg;       // log2(n)
  int np;       // n + 1
  T* u;
  T* b;
  T* ua;        // Chebyshev smoothing: second iterate buffer and the step direction
  T* d;
};

// One colour of a red-black sweep: items are (p, j[, l]) with i = 2p + 1 or 2p + 2, decoded
// with shifts; rows 0 and n and out-of-range i are skipped.
template <typename T, int D>
__device__ __forceinline__ void cta_rbgs(const CoarseLevel<T, D>& L, int colour, T bscale, T inv2d) {
  const int n = L.n, np = L.np, lgh = L.lg - 1;
  const int total = D == 2 ? (n << lgh) : (n << (lgh + L.lg));
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int p = t & ((1 << lgh) - 1);
    const int j = (t >> lgh) & (n - 1);
    const int l = D == 3 ? (t >> (lgh + L.lg)) : 0;
    if (j == 0 || (D == 3 && l == 0)) continue;
    const int par = (colour + j + l) & 1;
    const int i = par ? 2 * p + 1 : 2 * p + 2;
    if (i > n - 1) continue;
    const int c = (l * np + j) * np + i;
    T s = (L.u[c - 1] + L.u[c + 1]) + (L.u[c - np] + L.u[c + np]);
    if (D == 3) s += L.u[c - np * np] + L.u[c + np * np];
    L.u[c] = (L.b[c] * bscale + s) * inv2d;
  }
}

// The buffer in which a Chebyshev step 0 taken from a zero start (by the code that writes
// the level's b) leaves the iterate, so that steps 1..steps-1 end in L.u.
template <typename T, int D>
__device__ __forceinline__ T* cta_cheb_start(const CoarseLevel<T, D>& L, int steps) {
  return ((steps - 1) & 1) ? L.ua : L.u;
}

// Chebyshev-Jacobi steps k0..steps-1 on level L (colour-free: every interior node per step,
// the iterate alternating between u and ua); they start in L.u (k0 = 0) or in
// cta_cheb_start(L, steps) with d set (k0 = 1), and the result ends in L.u.
template <typename T, int D>
__device__ void cta_cheb(const CoarseLevel<T, D>& L, const ChebCoef& cf, int steps, T bscale, T inv2d, int k0 = 0) {
  const int n = L.n, np = L.np, lg = L.lg;
  const int total = D == 2 ? (1 << (2 * lg)) : (1 << (3 * lg));
  T* u = k0 ? cta_cheb_start(L, steps) : L.u;
  T* ua = u == L.u ? L.ua : L.u;
  for (int k = k0; k < steps; ++k) {
    const T cd = (T)cf.cd[k], cr = (T)cf.cr[k];
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int i = t & (n - 1), j = (t >> lg) & (n - 1), l = D == 3 ? (t >> (2 * lg)) : 0;
      if (i == 0 || j == 0 || (D == 3 && l == 0)) continue;
      const int c = (l * np + j) * np + i;
      T s = (u[c - 1] + u[c + 1]) + (u[c - np] + u[c + np]);
      if (D == 3) s += u[c - np * np] + u[c + np * np];
      const T z = (L.b[c] * bscale + s) * inv2d - u[c];
      const T dn = k == 0 ? cr * z : cd * L.d[c] + cr * z;
      L.d[c] = dn;
      ua[c] = u[c] + dn;
    }
    __syncthreads();
    T* t2 = u;
    u = ua;
    ua = t2;
  }
  if (u != L.u) {
    const int nodes = D == 2 ? np * np : np * np * np;
    for (int c = threadIdx.x; c < nodes; c += blockDim.x) L.u[c] = u[c];
    __syncthreads();
  }
}

template <typename T, int D>
__device__ __forceinline__ T cta_res(const CoarseLevel<T, D>& L, int c, T sigma) {
  const int np = L.np;
  T s = (L.u[c - 1] + L.u[c + 1]) + (L.u[c - np] + L.u[c + np]);
  if (D == 3) s += L.u[c - np * np] + L.u[c + np * np];
  return L.b[c] - sigma * (T(2 * D) * L.u[c] - s);
}

// zero_start: the top level's u is zero on entry (a correction from zero): it is not read,
// and with Chebyshev smoothing the top level's step 0 (pointwise from zero) is taken while b
// is loaded.  Below the top level the restriction takes the coarse level's step 0 the same
// way.  The FP32 cycle's level-1 solve uses an FP32 copy of A_1^{-1} (Ainv32), staged in
// shared memory while the top level loads; the FP64 cycle reads the FP64 A_1^{-1}.
template <typename T, int D>
__device__ __forceinline__ void k_vcycle_coarse_body(T* __restrict__ ug, const T* __restrict__ bg, int n0, int jtop, int nu_pre,
                                int nu_post, const double* __restrict__ Ainv, const float* __restrict__ Ainv32,
                                int cheb, const ChebCoef& cf, int zero_start) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  // level descriptors, the same for every thread: in shared memory (a per-thread copy would
  // be local memory, 1024 copies of it)
  __shared__ CoarseLevel<T, D> L[8];
  __shared__ int ai_off;
  constexpr bool kStageInv = sizeof(T) == sizeof(float);
  if (threadIdx.x == 0) {
    int off = 0;
    for (int j = 1; j <= jtop; ++j) {
      const int n = n0 << (j - 1);
      const int np = n + 1;
      const int nodes = D == 2 ? np * np : np * np * np;
      L[j - 1].n = n;
      L[j - 1].lg = 31 - __clz(n);
      L[j - 1].np = np;
      L[j - 1].u = sm + off;
      L[j - 1].b = sm + off + nodes;
      L[j - 1].ua = cheb ? sm + off + 2 * nodes : nullptr;
      L[j - 1].d = cheb ? sm + off + 3 * nodes : nullptr;
      off += (cheb ? 4 : 2) * nodes;
    }
    ai_off = off;
  }
  __syncthreads();
  float* ai = kStageInv ? reinterpret_cast<float*>(sm + ai_off) : nullptr;   // staged FP32 A_1^{-1}
  const T inv2d = T(1) / T(2 * D);
  const int m1 = n0 - 1;
  const int N1 = D == 2 ? m1 * m1 : m1 * m1 * m1;
  {
    const CoarseLevel<T, D>& top = L[jtop - 1];
    const int np = top.np;
    const int nodes = D == 2 ? np * np : np * np * np;
    // top level: b, and u (or, from a zero start, u = 0 or the first Chebyshev step); the
    // FP32 cycle also stages A_1^{-1}.  Every global load of a thread is issued before the
    // first store, so the phase costs about one memory latency.
    const bool first_top = cheb && zero_start && nu_pre >= 1 && jtop >= 2;
    const T e0 = T(cf.cr[0]) * (D == 2 ? T(1) : T(top.n)) * inv2d;   // step 0 from zero: cr_0 D^{-1} b
    T* ustart = first_top ? cta_cheb_start(top, nu_pre) : top.u;
    const int nai = kStageInv ? N1 * N1 : 0;
    for (int i0 = threadIdx.x; i0 < nodes || i0 < nai; i0 += 4 * blockDim.x) {
      T bv[4], uv[4];
      float av[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = i0 + r * blockDim.x;
        bv[r] = i < nodes ? bg[i] : T(0);
        uv[r] = (i < nodes && !zero_start) ? ug[i] : T(0);
        av[r] = i < nai ? __ldg(&Ainv32[i]) : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = i0 + r * blockDim.x;
        if (i < nai) ai[i] = av[r];
        if (i >= nodes) continue;
        top.b[i] = bv[r];
        top.u[i] = uv[r];
        if (first_top) {
          const int x = i % np, y = (i / np) % np, z = D == 3 ? i / (np * np) : 1;
          const bool inner = x > 0 && x < np - 1 && y > 0 && y < np - 1 && (D == 2 || (z > 0 && z < np - 1));
          const T e = inner ? e0 * bv[r] : T(0);
          ustart[i] = e;
          top.d[i] = e;
        }
      }
    }
    // lower levels: zero (boundary rings stay zero); the other Chebyshev buffers too
    for (int j = 1; j <= jtop; ++j) {
      const CoarseLevel<T, D>& Lj = L[j - 1];
      const int nn = D == 2 ? Lj.np * Lj.np : Lj.np * Lj.np * Lj.np;
      if (j < jtop)
        for (int i = threadIdx.x; i < 2 * nn; i += blockDim.x) Lj.u[i] = T(0);
      if (cheb) {
        if (j < jtop) {
          for (int i = threadIdx.x; i < 2 * nn; i += blockDim.x) Lj.ua[i] = T(0);
        } else {
          T* other = ustart == top.u ? top.ua : top.u;   // the top level's u, d and start are set above
          for (int i = threadIdx.x; i < nn; i += blockDim.x) {
            if (other == top.ua) top.ua[i] = T(0);
            if (!first_top) top.d[i] = T(0);
          }
        }
      }
    }
  }
  __syncthreads();
  // descend
  for (int j = jtop; j >= 2; --j) {
    const CoarseLevel<T, D>& F = L[j - 1];
    const CoarseLevel<T, D>& C = L[j - 2];
    const T bscale = D == 2 ? T(1) : T(F.n);
    const T sigma = D == 2 ? T(1) : T(1) / T(F.n);
    if (cheb) {
      // step 0 was taken by the load (top level from zero) or by the restriction (below)
      const bool started = nu_pre >= 1 && (j < jtop || zero_start);
      cta_cheb<T, D>(F, cf, nu_pre, bscale, inv2d, started ? 1 : 0);
    } else {
      for (int it = 0; it < nu_pre; ++it) {
        cta_rbgs<T, D>(F, 0, bscale, inv2d);
        __syncthreads();
        cta_rbgs<T, D>(F, 1, bscale, inv2d);
        __syncthreads();
      }
    }
    // b_c = P^T (b - A u), u_c = 0 -- or, when the coarse level is smoothed by Chebyshev
    // steps, its step 0 from zero: u_c = d_c = cr_0 D^{-1} b_c in the start buffer.  Items
    // (I, J[, K]) over [0, n_c)^d, boundary skipped.
    const int lgc = C.lg;
    const int total = D == 2 ? (1 << (2 * lgc)) : (1 << (3 * lgc));
    const bool first_c = cheb && nu_pre >= 1 && j - 1 >= 2;
    const T e0c = T(cf.cr[0]) * (D == 2 ? T(1) : T(C.n)) * inv2d;
    T* ucs = first_c ? cta_cheb_start(C, nu_pre) : C.u;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int I = t & (C.n - 1), J = (t >> lgc) & (C.n - 1), K = D == 3 ? (t >> (2 * lgc)) : 0;
      if (I == 0 || J == 0 || (D == 3 && K == 0)) continue;
      const int np = F.np;
      const int Fc = ((2 * K) * np + 2 * J) * np + 2 * I;
      T r = cta_res<T, D>(F, Fc, sigma);
      T e = (cta_res<T, D>(F, Fc + 1, sigma) + cta_res<T, D>(F, Fc - 1, sigma)) +
            (cta_res<T, D>(F, Fc + np, sigma) + cta_res<T, D>(F, Fc - np, sigma)) +
            (cta_res<T, D>(F, Fc + np + 1, sigma) + cta_res<T, D>(F, Fc - np - 1, sigma));
      if (D == 3) {
        const int pl = np * np;
        const int o[4] = {pl, 1 + pl, np + pl, 1 + np + pl};
#pragma unroll
        for (int q = 0; q < 4; ++q) e += cta_res<T, D>(F, Fc + o[q], sigma) + cta_res<T, D>(F, Fc - o[q], sigma);
      }
      const int cc = (K * C.np + J) * C.np + I;
      const T bv = r + T(0.5) * e;
      C.b[cc] = bv;
      if (first_c) {
        ucs[cc] = e0c * bv;
        C.d[cc] = e0c * bv;
      } else {
        C.u[cc] = T(0);
      }
    }
    __syncthreads();
  }
  // level 1: u_1 = A_1^{-1} b_1 in FP64; b_1 staged as FP64 in the (now unused) level-1 u
  // slots is not possible for FP32 levels, so it goes to a small shared array
  {
    __shared__ double b1[kMaxCoarseN];
    __shared__ int off1[kMaxCoarseN];
    const CoarseLevel<T, D>& C = L[0];
    const int m = C.n - 1;
    const int N = D == 2 ? m * m : m * m * m;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
      const int i = c % m + 1, j = (c / m) % m + 1, l = D == 3 ? c / (m * m) + 1 : 0;
      off1[c] = (l * C.np + j) * C.np + i;
      b1[c] = (double)C.b[off1[c]];
    }
    __syncthreads();
    // row r: lanes of one warp split the columns (row r of the symmetric A_1^{-1} is read
    // contiguously), then a shuffle sum (fixed order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < N; r += nw) {
      if (kStageInv) {
        float acc = 0.f;
        for (int c = lane; c < N; c += 32) acc = fmaf(ai[r * N + c], (float)b1[c], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) C.u[off1[r]] = (T)acc;
      } else {
        double acc = 0.0;
        for (int c = lane; c < N; c += 32) acc = fma(__ldg(&Ainv[(long long)r * N + c]), b1[c], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) C.u[off1[r]] = (T)acc;
      }
    }
    __syncthreads();
  }
  // ascend
  for (int j = 2; j <= jtop; ++j) {
    const CoarseLevel<T, D>& F = L[j - 1];
    const CoarseLevel<T, D>& C = L[j - 2];
    const T bscale = D == 2 ? T(1) : T(F.n);
    const int lgf = F.lg;
    const int total = D == 2 ? (1 << (2 * lgf)) : (1 << (3 * lgf));
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int i = t & (F.n - 1), jj = (t >> lgf) & (F.n - 1), l = D == 3 ? (t >> (2 * lgf)) : 0;
      if (i == 0 || jj == 0 || (D == 3 && l == 0)) continue;
      const int a = ((l >> 1) * C.np + (jj >> 1)) * C.np + (i >> 1);
      const int z = (((l + 1) >> 1) * C.np + ((jj + 1) >> 1)) * C.np + ((i + 1) >> 1);
      F.u[(l * F.np + jj) * F.np + i] += T(0.5) * (C.u[a] + C.u[z]);
    }
    __syncthreads();
    if (cheb) {
      cta_cheb<T, D>(F, cf, nu_post, bscale, inv2d);
    } else {
      for (int it = 0; it < nu_post; ++it) {
        cta_rbgs<T, D>(F, 1, bscale, inv2d);
        __syncthreads();
        cta_rbgs<T, D>(F, 0, bscale, inv2d);
        __syncthreads();
      }
    }
  }
  {
    const CoarseLevel<T, D>& top = L[jtop - 1];
    const int nodes = D == 2 ? top.np * top.np : top.np * top.np * top.np;
    for (int i = threadIdx.x; i < nodes; i += blockDim.x) ug[i] = top.u[i];
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(1024) k_vcycle_coarse(T* __restrict__ ug, const T* __restrict__ bg, int n0, int jtop, int nu_pre,
                                int nu_post, const double* __restrict__ Ainv, const float* __restrict__ Ainv32,
                                int cheb, const __grid_constant__ ChebCoef cf, int zero_start) { pdl_start(); k_vcycle_coarse_body<T, D>(ug, bg, n0, jtop, nu_pre, nu_post, Ainv, Ainv32, cheb, cf, zero_start); }

}  // namespace

// ============================================================================ launchers

template <typename T>
cudaError_t launch_rbgs(int dim, LevelGeo g, T* u, const T* b, int colour, cudaStream_t s, const VarCoef* vc) {
  const int n = g.n;
  const unsigned gx = cdiv(n / 2, kBlock);
  if (vc && vc->a64) {
    const int ls = vc_ls(*vc, n);
    if (dim == 2)
      launch_k(k_rbgs_vc<T, 2>, dim3(gx, n - 1), kBlock, 0, s, u, b, n, colour, ls, *vc);
    else
      launch_k(k_rbgs_vc<T, 3>, dim3(gx, n - 1, n - 1), kBlock, 0, s, u, b, n, colour, ls, *vc);
    return cudaGetLastError();
  }
  if (dim == 2) {
    launch_k(k_rbgs2<T>, dim3(gx, n - 1), kBlock, 0, s, u, b, n, colour);
  } else {
    launch_k(k_rbgs3<T>, dim3(gx, n - 1, n - 1), kBlock, 0, s, u, b, n, colour, T(n), T(1.0 / 6.0));
  }
  return cudaGetLastError();
}

template <typename TF, typename TC>
cudaError_t launch_residual_restrict(int dim, LevelGeo gf, const TF* u_f, const TF* b_f, LevelGeo gc, TC* b_c,
                                     TC* u_c, cudaStream_t s, TC* d_c, double e0, const VarCoef* vc) {
  const int nc = gc.n;
  const unsigned gx = cdiv(nc - 1, kBlock);
  if (vc && vc->a64) {
    if (d_c) return cudaErrorInvalidValue;   // Chebyshev smoothing does not take A(x)
    const int ls = vc_ls(*vc, gf.n);
    if (dim == 2)
      launch_k(k_resrestrict_vc<TF, TC, 2>, dim3(gx, nc - 1), kBlock, 0, s, u_f, b_f, gf.n, ls, *vc, b_c, u_c, nc);
    else
      launch_k(k_resrestrict_vc<TF, TC, 3>, dim3(gx, nc - 1, nc - 1), kBlock, 0, s, u_f, b_f, gf.n, ls, *vc, b_c, u_c, nc);
    return cudaGetLastError();
  }
  if (dim == 2) {
    const int S = rr_strip(nc);
    const dim3 grid(gx, cdiv(nc - 1, S));
    if (S == 1)
      launch_k(k_resrestrict2<TF, TC, 1>, grid, kBlock, 0, s, u_f, b_f, gf.n, b_c, u_c, nc, d_c, TC(e0));
    else if (S == 2)
      launch_k(k_resrestrict2<TF, TC, 2>, grid, kBlock, 0, s, u_f, b_f, gf.n, b_c, u_c, nc, d_c, TC(e0));
    else
      launch_k(k_resrestrict2<TF, TC, 4>, grid, kBlock, 0, s, u_f, b_f, gf.n, b_c, u_c, nc, d_c, TC(e0));
  } else {
    launch_k(k_resrestrict3<TF, TC>, dim3(gx, nc - 1, nc - 1), kBlock, 0, s, u_f, b_f, gf.n, TF(1.0) / TF(gf.n), b_c,
                                                                        u_c, nc, d_c, TC(e0));
  }
  return cudaGetLastError();
}

cudaError_t launch_residual_to_f32(int dim, LevelGeo g, const double* u, const double* b, float* r32, float* e32,
                                   cudaStream_t s, float* d32, double e0, const VarCoef* vc) {
  const int n = g.n;
  const unsigned gx = cdiv(n + 1, kBlock);
  if (vc && vc->a64) {
    if (d32) return cudaErrorInvalidValue;
    const int ls = vc_ls(*vc, n);
    if (dim == 2)
      launch_k(k_residual_vc<2>, dim3(gx, n + 1), kBlock, 0, s, u, b, n, ls, *vc, nullptr, r32, e32);
    else
      launch_k(k_residual_vc<3>, dim3(gx, n + 1, n + 1), kBlock, 0, s, u, b, n, ls, *vc, nullptr, r32, e32);
    return cudaGetLastError();
  }
  if (dim == 2)
    launch_k(k_residual2, dim3(gx, n + 1), kBlock, 0, s, u, b, n, nullptr, r32, e32, d32, (float)e0);
  else
    launch_k(k_residual3, dim3(gx, n + 1, n + 1), kBlock, 0, s, u, b, n, 1.0 / n, nullptr, r32, e32, d32, (float)e0);
  return cudaGetLastError();
}

cudaError_t launch_residual(int dim, LevelGeo g, const double* u, const double* b, double* r, cudaStream_t s,
                            const VarCoef* vc) {
  const int n = g.n;
  const unsigned gx = cdiv(n + 1, kBlock);
  if (vc && vc->a64) {
    const int ls = vc_ls(*vc, n);
    if (dim == 2)
      launch_k(k_residual_vc<2>, dim3(gx, n + 1), kBlock, 0, s, u, b, n, ls, *vc, r, nullptr, nullptr);
    else
      launch_k(k_residual_vc<3>, dim3(gx, n + 1, n + 1), kBlock, 0, s, u, b, n, ls, *vc, r, nullptr, nullptr);
    return cudaGetLastError();
  }
  if (dim == 2)
    launch_k(k_residual2, dim3(gx, n + 1), kBlock, 0, s, u, b, n, r, nullptr, nullptr, nullptr, 0.0f);
  else
    launch_k(k_residual3, dim3(gx, n + 1, n + 1), kBlock, 0, s, u, b, n, 1.0 / n, r, nullptr, nullptr, nullptr, 0.0f);
  return cudaGetLastError();
}

template <typename TF, typename TC>
cudaError_t launch_prolong(int dim, LevelGeo gc, const TC* e_c, LevelGeo gf, TF* u_f, int add, cudaStream_t s) {
  const int nf = gf.n;
  const unsigned gx = cdiv(nf - 1, kBlock);
  if (dim == 2)
    launch_k(k_prolong2<TF, TC>, dim3(gx, nf - 1), kBlock, 0, s, e_c, gc.n, u_f, nf, add);
  else
    launch_k(k_prolong3<TF, TC>, dim3(gx, nf - 1, nf - 1), kBlock, 0, s, e_c, gc.n, u_f, nf, add);
  return cudaGetLastError();
}

cudaError_t launch_add_f32(LevelGeo g, int dim, double* u, const float* e32, cudaStream_t s) {
  (void)dim;
  launch_k(k_add_f32, cdiv(g.nodes, 256), 256, 0, s, u, e32, g.nodes);
  return cudaGetLastError();
}

cudaError_t launch_nonlinear_rhs(int dim, LevelGeo g, const double* u, const double* gn, double* b, int kind,
                                 double a, cudaStream_t s) {
  const double h = 1.0 / g.n;
  const double w = dim == 2 ? h * h : h * h * h;
  const unsigned gx = cdiv(g.n + 1, kBlock);
  launch_k(k_nonlinear_rhs, dim3(gx, g.n + 1, dim == 3 ? g.n + 1 : 1), kBlock, 0, s, u, gn, b, g.n, dim, kind, a, w);
  return cudaGetLastError();
}

cudaError_t launch_copy(const double* src, double* dst, long long n, cudaStream_t s) {
  launch_k(k_copy, cdiv(n, 256), 256, 0, s, src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve_f64(int dim, LevelGeo g1, const double* Ainv, const double* b, double* u,
                                    cudaStream_t s) {
  const int m = g1.n - 1;
  const int N = (int)ipow(m, dim);
  launch_k(k_coarse_solve<double>, 1, 64, N * sizeof(double), s, Ainv, b, u, m, N, dim);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve_f32(int dim, LevelGeo g1, const double* Ainv, const float* b, float* u,
                                    cudaStream_t s) {
  const int m = g1.n - 1;
  const int N = (int)ipow(m, dim);
  launch_k(k_coarse_solve<float>, 1, 64, N * sizeof(double), s, Ainv, b, u, m, N, dim);
  return cudaGetLastError();
}

template <typename T>
size_t coarse_cycle_smem(int dim, int n0, int jtop, bool cheb) {
  size_t tot = 0;
  for (int j = 1; j <= jtop; ++j) {
    const long long np = (long long)(n0 << (j - 1)) + 1;
    tot += (cheb ? 4 : 2) * (size_t)ipow(np, dim);
  }
  // the FP32 cycle stages its FP32 A_1^{-1}
  const size_t n1 = (size_t)ipow(n0 - 1, dim);
  return tot * sizeof(T) + (sizeof(T) == sizeof(float) ? n1 * n1 * sizeof(float) : 0);
}

template <typename T>
cudaError_t launch_coarse_cycle(int dim, int n0, int jtop, T* u, const T* b, int nu_pre, int nu_post,
                                const double* Ainv, const float* Ainv32, const ChebCoef* cheb, bool zero_start,
                                cudaStream_t s) {
  if (sizeof(T) == sizeof(float) && !Ainv32) return cudaErrorInvalidValue;
  if (cheb && (nu_pre > kMaxCheb || nu_post > kMaxCheb)) return cudaErrorInvalidValue;
  const size_t smem = coarse_cycle_smem<T>(dim, n0, jtop, cheb != nullptr);
  const ChebCoef cf = cheb ? *cheb : ChebCoef{};
  cudaError_t e;
  if (dim == 2) {
    if ((e = raise_dyn_smem((const void*)k_vcycle_coarse<T, 2>, smem)) != cudaSuccess) return e;
    launch_k(k_vcycle_coarse<T, 2>, 1, 1024, smem, s, u, b, n0, jtop, nu_pre, nu_post, Ainv, Ainv32, cheb ? 1 : 0, cf,
                                                 zero_start ? 1 : 0);
  } else {
    if ((e = raise_dyn_smem((const void*)k_vcycle_coarse<T, 3>, smem)) != cudaSuccess) return e;
    launch_k(k_vcycle_coarse<T, 3>, 1, 1024, smem, s, u, b, n0, jtop, nu_pre, nu_post, Ainv, Ainv32, cheb ? 1 : 0, cf,
                                                 zero_start ? 1 : 0);
  }
  return cudaGetLastError();
}

ChebCoef cheb_coefficients() {
  // lmax = 2 bounds the spectrum of D^{-1}A for the 2d+1-point stiffness; the smoother
  // targets [lmax/4, lmax]
  const double lmax = 2.0, lmin = lmax / 4.0;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sig = theta / delta;
  ChebCoef c{};
  c.cd[0] = 0.0;
  c.cr[0] = 1.0 / theta;
  double rho = 1.0 / sig;
  for (int k = 1; k < kMaxCheb; ++k) {
    const double rn = 1.0 / (2.0 * sig - rho);
    c.cd[k] = rn * rho;
    c.cr[k] = 2.0 * rn / delta;
    rho = rn;
  }
  return c;
}

// Launch shapes of the Chebyshev step kernel picked by the autotuner (fmg_autotune), per
// device, dimension, cells per side and element size; absent entries use the default rule.
namespace {
std::mutex g_shape_mu;
std::map<std::tuple<int, int, int, int>, ChebShape> g_shapes;

ChebShape default_cheb_shape(int dim, int n) {
  const unsigned gx = cdiv(n - 1, kBlock);
  const unsigned plane = dim == 2 ? gx : gx * (unsigned)(n - 1);
  // the longest strip that still leaves at least 1024 blocks (small levels: one node each)
  int strip = kChebStrip;
  while (strip > 1 && (long long)plane * cdiv(n - 1, strip) < 1024) strip >>= 1;
  return ChebShape{kBlock, strip};
}
}  // namespace

ChebShape cheb_shape(int dim, int n, int elem_bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_shape_mu);
  auto it = g_shapes.find(std::make_tuple(dev, dim, n, elem_bytes));
  return it != g_shapes.end() ? it->second : default_cheb_shape(dim, n);
}

bool cheb_shape_tuned(int dim, int n, int elem_bytes, ChebShape* out) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_shape_mu);
  auto it = g_shapes.find(std::make_tuple(dev, dim, n, elem_bytes));
  if (it == g_shapes.end()) return false;
  if (out) *out = it->second;
  return true;
}

void set_cheb_shape(int dim, int n, int elem_bytes, ChebShape sh) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_shape_mu);
  g_shapes[std::make_tuple(dev, dim, n, elem_bytes)] = sh;
}

template <typename T>
cudaError_t launch_cheb_shaped(int dim, LevelGeo g, const T* u, T* uo, T* d, const T* b, double cd, double cr,
                               bool first, ChebShape sh, cudaStream_t s, const T* ec) {
  const int n = g.n;
  if (sh.block < 32 || sh.block > 1024 || (sh.block & 31) || sh.strip < 1 || sh.strip > kChebStrip)
    return cudaErrorInvalidValue;
  const unsigned gx = cdiv(n - 1, sh.block);
  const unsigned gs = cdiv(n - 1, sh.strip);
  const dim3 grid = dim == 2 ? dim3(gx, gs) : dim3(gx, n - 1, gs);
  const T bs = dim == 2 ? T(1) : T(n);
  const int f = first ? 1 : 0;
  if (dim == 2 && ec)
    launch_k(k_cheb<T, 2, true>, grid, sh.block, 0, s, u, uo, d, b, n, bs, T(cd), T(cr), f, sh.strip, ec);
  else if (dim == 2)
    launch_k(k_cheb<T, 2, false>, grid, sh.block, 0, s, u, uo, d, b, n, bs, T(cd), T(cr), f, sh.strip, ec);
  else if (ec)
    launch_k(k_cheb<T, 3, true>, grid, sh.block, 0, s, u, uo, d, b, n, bs, T(cd), T(cr), f, sh.strip, ec);
  else
    launch_k(k_cheb<T, 3, false>, grid, sh.block, 0, s, u, uo, d, b, n, bs, T(cd), T(cr), f, sh.strip, ec);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cheb(int dim, LevelGeo g, const T* u, T* uo, T* d, const T* b, double cd, double cr, bool first,
                        cudaStream_t s, const T* ec) {
  return launch_cheb_shaped<T>(dim, g, u, uo, d, b, cd, cr, first, cheb_shape(dim, g.n, (int)sizeof(T)), s, ec);
}

cudaError_t launch_cheb_add64(int dim, LevelGeo g, const float* u, const float* d, const float* b, double* u64,
                              double cd, double cr, bool first, cudaStream_t s, bool u_ff) {
  const int n = g.n;
  const ChebShape sh = cheb_shape(dim, n, 4);
  const unsigned gx = cdiv(n - 1, sh.block);
  const unsigned gs = cdiv(n - 1, sh.strip);
  const dim3 grid = dim == 2 ? dim3(gx, gs) : dim3(gx, n - 1, gs);
  const float bs = dim == 2 ? 1.0f : (float)n;
  const int f = first ? 1 : 0;
  if (dim == 2 && u_ff)
    launch_k(k_cheb_add64<2, true>, grid, sh.block, 0, s, u, d, b, u64, n, bs, (float)cd, (float)cr, f, sh.strip);
  else if (dim == 2)
    launch_k(k_cheb_add64<2, false>, grid, sh.block, 0, s, u, d, b, u64, n, bs, (float)cd, (float)cr, f, sh.strip);
  else if (u_ff)
    launch_k(k_cheb_add64<3, true>, grid, sh.block, 0, s, u, d, b, u64, n, bs, (float)cd, (float)cr, f, sh.strip);
  else
    launch_k(k_cheb_add64<3, false>, grid, sh.block, 0, s, u, d, b, u64, n, bs, (float)cd, (float)cr, f, sh.strip);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* src, float* dst, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  launch_k(k_to_f32, cdiv(n, 256), 256, 0, s, src, dst, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_t(const T* src, T* dst, long long n, cudaStream_t s) {
  launch_k(k_copy_t<T>, cdiv(n, 256), 256, 0, s, src, dst, n);
  return cudaGetLastError();
}

template size_t coarse_cycle_smem<double>(int, int, int, bool);
template size_t coarse_cycle_smem<float>(int, int, int, bool);
template cudaError_t launch_coarse_cycle<double>(int, int, int, double*, const double*, int, int, const double*,
                                                 const float*, const ChebCoef*, bool, cudaStream_t);
template cudaError_t launch_coarse_cycle<float>(int, int, int, float*, const float*, int, int, const double*,
                                                const float*, const ChebCoef*, bool, cudaStream_t);
template cudaError_t launch_cheb<double>(int, LevelGeo, const double*, double*, double*, const double*, double, double,
                                         bool, cudaStream_t, const double*);
template cudaError_t launch_cheb<float>(int, LevelGeo, const float*, float*, float*, const float*, double, double, bool,
                                        cudaStream_t, const float*);
template cudaError_t launch_cheb_shaped<double>(int, LevelGeo, const double*, double*, double*, const double*, double,
                                                double, bool, ChebShape, cudaStream_t, const double*);
template cudaError_t launch_cheb_shaped<float>(int, LevelGeo, const float*, float*, float*, const float*, double,
                                               double, bool, ChebShape, cudaStream_t, const float*);
template cudaError_t launch_copy_t<double>(const double*, double*, long long, cudaStream_t);
template cudaError_t launch_copy_t<float>(const float*, float*, long long, cudaStream_t);
template cudaError_t launch_rbgs<double>(int, LevelGeo, double*, const double*, int, cudaStream_t, const VarCoef*);
template cudaError_t launch_rbgs<float>(int, LevelGeo, float*, const float*, int, cudaStream_t, const VarCoef*);
template cudaError_t launch_residual_restrict<double, double>(int, LevelGeo, const double*, const double*, LevelGeo,
                                                              double*, double*, cudaStream_t, double*, double,
                                                              const VarCoef*);
template cudaError_t launch_residual_restrict<float, float>(int, LevelGeo, const float*, const float*, LevelGeo,
                                                            float*, float*, cudaStream_t, float*, double,
                                                            const VarCoef*);
template cudaError_t launch_prolong<double, double>(int, LevelGeo, const double*, LevelGeo, double*, int,
                                                    cudaStream_t);
template cudaError_t launch_prolong<float, float>(int, LevelGeo, const float*, LevelGeo, float*, int, cudaStream_t);

}  // namespace fmg

namespace fmg {

cudaError_t raise_dyn_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[std::make_pair(dev, kernel)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}


// The 2D kernels of the solve's cycles, for phase-batched launches.
void phase_kernels_stencil(std::vector<PhaseKernel>& out) {
  out.push_back(phase_kernel<&k_rbgs2_body<float>, kBlock, 1>(&k_rbgs2<float>));
  out.push_back(phase_kernel<&k_rbgs2_body<double>, kBlock, 1>(&k_rbgs2<double>));
  out.push_back(phase_kernel<&k_cheb_body<float, 2, false>, 512, 1>(&k_cheb<float, 2, false>));
  out.push_back(phase_kernel<&k_cheb_body<float, 2, true>, 512, 3>(&k_cheb<float, 2, true>));
  out.push_back(phase_kernel<&k_cheb_body<double, 2, false>, 512, 4>(&k_cheb<double, 2, false>));
  out.push_back(phase_kernel<&k_cheb_body<double, 2, true>, 512, 2>(&k_cheb<double, 2, true>));
  out.push_back(phase_kernel<&k_cheb_add64_body<2, true>, 512, 1>(&k_cheb_add64<2, true>));
  out.push_back(phase_kernel<&k_cheb_add64_body<2, false>, 512, 1>(&k_cheb_add64<2, false>));
  out.push_back(phase_kernel<&k_copy_t_body<float>, 256, 1>(&k_copy_t<float>));
  out.push_back(phase_kernel<&k_copy_t_body<double>, 256, 1>(&k_copy_t<double>));
  out.push_back(phase_kernel<&k_resrestrict2_body<float, float, 1>, kBlock, 8>(&k_resrestrict2<float, float, 1>));
  out.push_back(phase_kernel<&k_resrestrict2_body<float, float, 2>, kBlock, 8>(&k_resrestrict2<float, float, 2>));
  out.push_back(phase_kernel<&k_resrestrict2_body<float, float, 4>, kBlock, 8>(&k_resrestrict2<float, float, 4>));
  out.push_back(phase_kernel<&k_resrestrict2_body<double, double, 1>, kBlock, 6>(&k_resrestrict2<double, double, 1>));
  out.push_back(phase_kernel<&k_resrestrict2_body<double, double, 2>, kBlock, 6>(&k_resrestrict2<double, double, 2>));
  out.push_back(phase_kernel<&k_resrestrict2_body<double, double, 4>, kBlock, 6>(&k_resrestrict2<double, double, 4>));
  out.push_back(phase_kernel<&k_prolong2_body<float, float>, kBlock, 1>(&k_prolong2<float, float>));
  out.push_back(phase_kernel<&k_prolong2_body<double, double>, kBlock, 1>(&k_prolong2<double, double>));
  out.push_back(phase_kernel<&k_nonlinear_rhs_body, kBlock, 1>(&k_nonlinear_rhs));
  out.push_back(phase_kernel<&k_coarse_solve_body<float>, 64, 24>(&k_coarse_solve<float>));
  out.push_back(phase_kernel<&k_coarse_solve_body<double>, 64, 24>(&k_coarse_solve<double>));
  out.push_back(phase_kernel<&k_vcycle_coarse_body<float, 2>, 1024, 1>(&k_vcycle_coarse<float, 2>));
  out.push_back(phase_kernel<&k_vcycle_coarse_body<double, 2>, 1024, 1>(&k_vcycle_coarse<double, 2>));
}

}  // namespace fmg

// Fused FP32 multigrid-cycle kernels for the fine levels of the mixed-precision path (2D).
//
// One V-cycle level (Algorithm 3.1 step 1, eq. 3.5) in two launches instead of 2 nu + 2:
//   pre:  nu red-black sweeps from a zero initial guess (the correction equation of the
//         defect-correction loop, or a coarser level of the cycle, always starts at zero),
//         then b_c = P^T (b - A u) and u_c = 0 on the next coarser level;
//   post: u += P e_c, then nu black-red sweeps; on the cycle's top level the result is added
//         to the iterate (the update of the defect correction; FP64 in the ops, float-float in
//         a mixed solve) instead of being stored.
// Each block owns a 64 x 64 tile of fine nodes and works in shared memory on the tile plus
// a halo as wide as the sweeps' reach (2 nu, plus 2 for the residual and restriction), so
// neighbouring tiles are independent: every sweep is computed redundantly on the part of
// the halo it needs.  Inputs and outputs are different arrays (the level's two FP32
// buffers), so no block reads a value another block has already overwritten.  The
// arithmetic of every node update, residual and restriction sum is the same expression, in
// the same order, as in the per-step kernels, so both give identical results.
#include <cuda_runtime.h>

#include "fmg_ff.cuh"
#include "fmg_internal.cuh"
#include "fmg_phase.cuh"

namespace fmg {

namespace {

constexpr int kFT = 64;     // fine tile edge
constexpr int kFB = 256;    // threads per block

// 4-byte asynchronous global -> shared copy (no register staging, so a thread has all its
// copies in flight at once); src_size 0 zero-fills nodes outside the interior.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(saddr), "l"(gmem), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// One colour of a red-black sweep on the local square [lo, hi]^2 of a W x W shared tile
// whose local (0, 0) is global (gx0, gy0); only interior nodes (0 < g < n) change.  Threads
// form 8 rows of 32; each takes two rows at a time and two nodes of the colour per row,
// computing all four updates before storing any (no node of one colour reads another of the
// same colour, so the order does not matter).
template <int W>
__device__ __forceinline__ void tile_halfsweep(float* su, const float* sb, int lo, int hi, int colour, int gx0,
                                               int gy0, int n) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int xlo = max(lo, 1 - gx0), xhi = min(hi, n - 1 - gx0);
  const int ylo = max(lo, 1 - gy0), yhi = min(hi, n - 1 - gy0);
  for (int ly = ylo + ty; ly <= yhi; ly += 16) {
    float v[4];
    int c[4];
    bool h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = ly + 8 * (q >> 1);
      const int gy = gy0 + row;
      const int first = xlo + ((colour + gy + gx0 + xlo) & 1);
      const int lx = first + 2 * tx + 64 * (q & 1);
      h[q] = row <= yhi && lx <= xhi;
      c[q] = row * W + lx;
      v[q] = h[q] ? (sb[c[q]] + ((su[c[q] - 1] + su[c[q] + 1]) + (su[c[q] - W] + su[c[q] + W]))) * 0.25f : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (h[q]) su[c[q]] = v[q];
  }
}

template <int NU>
__device__ __forceinline__ void k_pre2_fused_body(const float* __restrict__ b, float* __restrict__ u_out,
                                                     float* __restrict__ bc, float* __restrict__ uc, int n) {
  constexpr int H = 2 * NU + 2;
  constexpr int W = kFT + 2 * H;
  extern __shared__ float sm[];
  float* su = sm;
  float* sb = su + W * W;
  float* sr = sb + W * W;  // residual on fine nodes [X0-1, X0+kFT-1]^2, (kFT+1)^2
  const int X0 = blockIdx.x * kFT, Y0 = blockIdx.y * kFT;
  const int gx0 = X0 - H, gy0 = Y0 - H;
  const long long np = n + 1;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int ly = ty; ly < W; ly += 8) {
    const int gy = gy0 + ly;
    for (int lx = tx; lx < W; lx += 32) {
      const int gx = gx0 + lx;
      const bool in = gx > 0 && gx < n && gy > 0 && gy < n;
      cp_async4(&sb[ly * W + lx], in ? b + ((long long)gy * np + gx) : b, in);
      su[ly * W + lx] = 0.f;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int s = 0; s < 2 * NU; ++s) {
    tile_halfsweep<W>(su, sb, s + 1, W - 2 - s, s & 1, gx0, gy0, n);
    __syncthreads();
  }
  // residual r = b - A u on [X0-1, X0+kFT-1]^2 (zero outside the interior)
  constexpr int R = kFT + 1;
  for (int ry = ty; ry < R; ry += 8) {
    const int gy = Y0 - 1 + ry;
    for (int rx = tx; rx < R; rx += 32) {
      const int gx = X0 - 1 + rx;
      float r = 0.f;
      if (gx > 0 && gx < n && gy > 0 && gy < n) {
        const int c = (gy - gy0) * W + (gx - gx0);
        r = sb[c] - (4.0f * su[c] - ((su[c - 1] + su[c + 1]) + (su[c - W] + su[c + W])));
      }
      sr[ry * R + rx] = r;
    }
  }
  __syncthreads();
  // b_c = P^T r, u_c = 0 on the coarse nodes of the tile
  const int nc = n >> 1;
  const long long cp = nc + 1;
  constexpr int C = kFT / 2;
  for (int cy = ty; cy < C; cy += 8) {
    const int J = Y0 / 2 + cy;
    const int cx = tx;
    const int I = X0 / 2 + cx;
    if (I < 1 || I > nc - 1 || J < 1 || J > nc - 1) continue;
    const int F = (2 * cy + 1) * R + (2 * cx + 1);
    const float r = sr[F];
    const float e = (sr[F + 1] + sr[F - 1]) + (sr[F + R] + sr[F - R]) + (sr[F + R + 1] + sr[F - R - 1]);
    bc[J * cp + I] = r + 0.5f * e;
    uc[J * cp + I] = 0.f;
  }
  // the smoothed tile
  for (int ty2 = ty; ty2 < kFT; ty2 += 8) {
    const int gy = Y0 + ty2;
    for (int tx2 = tx; tx2 < kFT; tx2 += 32) {
      const int gx = X0 + tx2;
      if (gx > 0 && gx < n && gy > 0 && gy < n) u_out[(long long)gy * np + gx] = su[(ty2 + H) * W + (tx2 + H)];
    }
  }
}

template <int NU>
__global__ void __launch_bounds__(kFB) k_pre2_fused(const float* __restrict__ b, float* __restrict__ u_out,
                                                     float* __restrict__ bc, float* __restrict__ uc, int n) { pdl_start(); k_pre2_fused_body<NU>(b, u_out, bc, uc, n); }

// MODE 0: the smoothed correction goes to u_out; 1: it is added to the FP64 iterate u64 (the
// ops' arrays); 2: it is added to the float-float iterate u64 (the solve's level data).
template <int NU, int MODE>
__device__ __forceinline__ void k_post2_fused_body(const float* __restrict__ u_in, const float* __restrict__ ec,
                                                      const float* __restrict__ b, float* __restrict__ u_out,
                                                      double* __restrict__ u64, int n) {
  constexpr int H = 2 * NU;
  constexpr int W = kFT + 2 * H;
  extern __shared__ float sm[];
  float* su = sm;
  float* sb = su + W * W;
  const int X0 = blockIdx.x * kFT, Y0 = blockIdx.y * kFT;
  const int gx0 = X0 - H, gy0 = Y0 - H;
  const long long np = n + 1;
  const long long cp = (n >> 1) + 1;
  // coarse correction tile: coarse nodes [gx0/2 - 1, gx0/2 + W/2 + 1) (floor/ceil of the fine tile)
  constexpr int CW = W / 2 + 2;
  float* se = sb + W * W;
  const int cx0 = (gx0 >> 1) - 1, cy0 = (gy0 >> 1) - 1;
  const int ncl = n >> 1;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int ly = ty; ly < W; ly += 8) {
    const int gy = gy0 + ly;
    for (int lx = tx; lx < W; lx += 32) {
      const int gx = gx0 + lx;
      const bool in = gx > 0 && gx < n && gy > 0 && gy < n;
      const long long g = (long long)gy * np + gx;
      cp_async4(&su[ly * W + lx], in ? u_in + g : u_in, in);
      cp_async4(&sb[ly * W + lx], in ? b + g : b, in);
    }
  }
  for (int cy = ty; cy < CW; cy += 8) {
    const int Y = cy0 + cy;
    for (int cx = tx; cx < CW; cx += 32) {
      const int X = cx0 + cx;
      const bool in = X >= 0 && X <= ncl && Y >= 0 && Y <= ncl;
      cp_async4(&se[cy * CW + cx], in ? ec + ((long long)Y * cp + X) : ec, in);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // u += P e_c on the interior nodes of the tile region
  for (int ly = ty; ly < W; ly += 8) {
    const int gy = gy0 + ly;
    for (int lx = tx; lx < W; lx += 32) {
      const int gx = gx0 + lx;
      if (gx > 0 && gx < n && gy > 0 && gy < n) {
        const float v = 0.5f * (se[((gy >> 1) - cy0) * CW + ((gx >> 1) - cx0)] +
                                se[(((gy + 1) >> 1) - cy0) * CW + (((gx + 1) >> 1) - cx0)]);
        su[ly * W + lx] = su[ly * W + lx] + v;
      }
    }
  }
  __syncthreads();
  for (int s = 0; s < 2 * NU; ++s) {
    tile_halfsweep<W>(su, sb, s + 1, W - 2 - s, 1 - (s & 1), gx0, gy0, n);
    __syncthreads();
  }
  for (int ty2 = ty; ty2 < kFT; ty2 += 8) {
    const int gy = Y0 + ty2;
    for (int tx2 = tx; tx2 < kFT; tx2 += 32) {
      const int gx = X0 + tx2;
      if (gx > 0 && gx < n && gy > 0 && gy < n) {
        const long long g = (long long)gy * np + gx;
        const float v = su[(ty2 + H) * W + (tx2 + H)];
        if (MODE == 2)
          ff_store(u64 + g, ff_add_f(ff_load(u64 + g), v));
        else if (MODE == 1)
          u64[g] += (double)v;
        else
          u_out[g] = v;
      }
    }
  }
}

template <int NU, int MODE>
__global__ void __launch_bounds__(kFB) k_post2_fused(const float* __restrict__ u_in, const float* __restrict__ ec,
                                                      const float* __restrict__ b, float* __restrict__ u_out,
                                                      double* __restrict__ u64, int n) { pdl_start(); k_post2_fused_body<NU, MODE>(u_in, ec, b, u_out, u64, n); }

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return raise_dyn_smem((const void*)kernel, bytes);
}

}  // namespace

bool fused_cycle_supported(int dim, int nu_pre, int nu_post) {
  return dim == 2 && nu_pre >= 1 && nu_pre <= 2 && nu_post >= 1 && nu_post <= 2;
}

cudaError_t launch_pre_fused(int dim, LevelGeo g, int nu, const float* b, float* u_out, float* bc, float* uc,
                             cudaStream_t s) {
  if (dim != 2) return cudaErrorInvalidValue;
  const unsigned t = (unsigned)((g.n + 1 + kFT - 1) / kFT);
  const dim3 grid(t, t);
  cudaError_t e;
  if (nu == 1) {
    constexpr int W = kFT + 2 * 4;
    const size_t smem = sizeof(float) * (2 * W * W + (kFT + 1) * (kFT + 1));
    if ((e = set_smem(k_pre2_fused<1>, smem)) != cudaSuccess) return e;
    launch_k(k_pre2_fused<1>, grid, kFB, smem, s, b, u_out, bc, uc, g.n);
  } else {
    constexpr int W = kFT + 2 * 6;
    const size_t smem = sizeof(float) * (2 * W * W + (kFT + 1) * (kFT + 1));
    if ((e = set_smem(k_pre2_fused<2>, smem)) != cudaSuccess) return e;
    launch_k(k_pre2_fused<2>, grid, kFB, smem, s, b, u_out, bc, uc, g.n);
  }
  return cudaGetLastError();
}

cudaError_t launch_post_fused(int dim, LevelGeo g, int nu, const float* u_in, const float* ec, const float* b,
                              float* u_out, double* u64_top, cudaStream_t s, bool u_ff) {
  const int mode = u64_top ? (u_ff ? 2 : 1) : 0;
  if (dim != 2) return cudaErrorInvalidValue;
  const unsigned t = (unsigned)((g.n + 1 + kFT - 1) / kFT);
  const dim3 grid(t, t);
  cudaError_t e;
  if (nu == 1) {
    constexpr int W = kFT + 2 * 2;
    const size_t smem = sizeof(float) * (2 * W * W + (W / 2 + 2) * (W / 2 + 2));
    if (mode == 2) {
      if ((e = set_smem(k_post2_fused<1, 2>, smem)) != cudaSuccess) return e;
      launch_k(k_post2_fused<1, 2>, grid, kFB, smem, s, u_in, ec, b, u_out, u64_top, g.n);
    } else if (mode == 1) {
      if ((e = set_smem(k_post2_fused<1, 1>, smem)) != cudaSuccess) return e;
      launch_k(k_post2_fused<1, 1>, grid, kFB, smem, s, u_in, ec, b, u_out, u64_top, g.n);
    } else {
      if ((e = set_smem(k_post2_fused<1, 0>, smem)) != cudaSuccess) return e;
      launch_k(k_post2_fused<1, 0>, grid, kFB, smem, s, u_in, ec, b, u_out, u64_top, g.n);
    }
  } else {
    constexpr int W = kFT + 2 * 4;
    const size_t smem = sizeof(float) * (2 * W * W + (W / 2 + 2) * (W / 2 + 2));
    if (mode == 2) {
      if ((e = set_smem(k_post2_fused<2, 2>, smem)) != cudaSuccess) return e;
      launch_k(k_post2_fused<2, 2>, grid, kFB, smem, s, u_in, ec, b, u_out, u64_top, g.n);
    } else if (mode == 1) {
      if ((e = set_smem(k_post2_fused<2, 1>, smem)) != cudaSuccess) return e;
      launch_k(k_post2_fused<2, 1>, grid, kFB, smem, s, u_in, ec, b, u_out, u64_top, g.n);
    } else {
      if ((e = set_smem(k_post2_fused<2, 0>, smem)) != cudaSuccess) return e;
      launch_k(k_post2_fused<2, 0>, grid, kFB, smem, s, u_in, ec, b, u_out, u64_top, g.n);
    }
  }
  return cudaGetLastError();
}


// The fused 2D FP32 red-black kernels, for phase-batched launches.
void phase_kernels_fused(std::vector<PhaseKernel>& out) {
  out.push_back(phase_kernel<&k_pre2_fused_body<1>, kFB, 8>(&k_pre2_fused<1>));
  out.push_back(phase_kernel<&k_pre2_fused_body<2>, kFB, 8>(&k_pre2_fused<2>));
  out.push_back(phase_kernel<&k_post2_fused_body<1, 0>, kFB, 8>(&k_post2_fused<1, 0>));
  out.push_back(phase_kernel<&k_post2_fused_body<1, 1>, kFB, 8>(&k_post2_fused<1, 1>));
  out.push_back(phase_kernel<&k_post2_fused_body<1, 2>, kFB, 8>(&k_post2_fused<1, 2>));
  out.push_back(phase_kernel<&k_post2_fused_body<2, 0>, kFB, 8>(&k_post2_fused<2, 0>));
  out.push_back(phase_kernel<&k_post2_fused_body<2, 1>, kFB, 8>(&k_post2_fused<2, 1>));
  out.push_back(phase_kernel<&k_post2_fused_body<2, 2>, kFB, 8>(&k_post2_fused<2, 2>));
}

}  // namespace fmg

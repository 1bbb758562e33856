// Internal declarations shared by the CUDA translation units of the solver.
//
// Geometry: level k of the nested hierarchy (Sec. 3, eq. 3.1) has n = (1/H) 2^(k-1) cells
// per side and (n+1)^d nodes, boundary included, stored x fastest.  The P1 stiffness of
// the right-triangle (2D) and Kuhn (3D) meshes is sigma * (2d-point Laplacian) with
// sigma = h^(d-2); the vertex quadrature weight of an interior node is w = h^d.
#pragma once

#include <cuda_runtime.h>

#include <utility>
#include <stdint.h>

#include <string>

#include "../../include/fmg.h"

namespace fmg {

constexpr int kMaxLevels = 24;
constexpr int kMaxAug = 64;          // N_H + 1 limit of the dense augmented system
constexpr int kMaxNewton = 64;

// Device status flags (mirrors fmg_stats.flags).
constexpr unsigned kFlagNewtonCap = 1u;
constexpr unsigned kFlagNonfinite = 2u;
constexpr unsigned kFlagDropped = 4u;
constexpr unsigned kFlagNotSPD = 8u;
constexpr unsigned kFlagTimeout = 16u;

// Programmatic dependent launch.  Every kernel of the solve starts with pdl_start(): it lets the
// next kernel on the stream be scheduled (launch_dependents) and then waits until the previous
// kernel has completed and its memory is visible (wait), before touching memory.  launch_k
// launches a kernel with programmatic stream serialization (grids up to kPdlMaxBlocks blocks),
// so that, in a captured graph, the launch of a kernel and the start of its blocks overlap its
// predecessor's last blocks; the results are those of plain serialization.  Without the
// attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_start() {
#if defined(__CUDA_ARCH__)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// Grids of more blocks launch without it: many waves hide the launch anyway, and a grid's blocks
// placed early into whichever SMs free first were measured to unbalance the largest 3D kernels
// (3D solve 4.17 ms with every grid, 4.00 with this limit, 4.03 with none; 2D 1.37, 1.37, 1.45).
constexpr long long kPdlMaxBlocks = 65536;

// Launches of this thread ask for programmatic serialization only while t_pdl is set.  A context
// that has the device to itself captures with it set; contexts that run side by side (batch
// branches, the request server) capture with it clear, since a grid that launches early holds
// the SM slots its waiting blocks sit in, which the other streams' kernels would use (served
// requests measured 20-30 % slower with it).
inline thread_local bool t_pdl = true;

struct PdlScope {
  bool saved;
  explicit PdlScope(bool on) : saved(t_pdl) { t_pdl = on; }
  ~PdlScope() { t_pdl = saved; }
};

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = t_pdl && (long long)grid.x * grid.y * grid.z <= kPdlMaxBlocks ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Small per-context device state (one allocation, part of the workspace).
struct DevState {
  unsigned int flags;
  int level1_iters;
  int newton_iters[32];
  double alpha[32];
  // grid barrier of the cooperative Newton kernel
  unsigned int bar_count;
  unsigned int bar_gen;
  int abort;
  int converged;
  // arrivals of a pass's blocks per coarse cell (the last block of a cell sums its partial
  // rows; it resets the count to zero)
  unsigned int cell_count[64];
  // current augmented iterate
  double alpha_cur;
  double pad[3];
};

struct LevelGeo {
  int n;          // cells per side
  int np;         // n + 1
  long long nodes;  // (n+1)^d
};

__host__ __device__ inline long long ipow(long long b, int e) {
  long long r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Variable SPD coefficient A(x) of -div(A grad u) (Sec. 2, eq. 2.1): diagonal and constant on
// each cell of T_H (nc cells per side), one row of d entries per cell, x fastest; a64 == nullptr
// means A = I.  On the right-triangle and Kuhn meshes a diagonal A couples a simplex's vertices
// only along its axis path edges, so the stiffness stays a (2d+1)-point stencil, with a weight
// per axis edge: in 2D an x edge from (i, j) bounds fine cells (i, j) and (i, j-1), a y edge from
// (i, j) cells (i, j) and (i-1, j), each through one triangle, so w = (A(c1) + A(c2)) / 2; in 3D
// an x edge from (i, j, l) is a path edge of 2 Kuhn tetrahedra of fine cubes (i, j, l) and
// (i, j-1, l-1) and of 1 of cubes (i, j-1, l) and (i, j, l-1) (y and z alike by symmetry), so
// w = (2 A(c1) + 2 A(c2) + A(c3) + A(c4)) / 6, the stiffness being h times these sums.  A fine
// cell (p, q[, r]) of a level with 2^ls fine cells per coarse cell lies in coarse cell
// (p >> ls, q >> ls[, r >> ls]).  With A = I every weight is 1.
struct VarCoef {
  const double* a64;   // FP64 entries, nullptr: A = I
  const float* a32;    // FP32 entries
  const double* aff;   // float-float entries (hi, lo) in 8-byte slots
  int nc;              // cells per side of T_H
};

template <int D>
__host__ __device__ __forceinline__ int coef_index(int nc, int cx, int cy, int cz, int axis) {
  return (D == 2 ? cy * nc + cx : (cz * nc + cy) * nc + cx) * D + axis;
}

// The weights of the 2d axis edges at node (i, j[, l]) of a level with 2^ls fine cells per
// coarse cell, in the order x-, x+, y-, y+ (, z-, z+), from the entries val(k) (an index into the
// table as coef_index gives it), combined by add(x, y) and scaled by half(x) (x / 2) or sixth(x)
// (x / 6): the precision-agnostic form the FP64, FP32 and float-float kernels share.
template <int D, typename V, typename Val, typename Add, typename Scale>
__host__ __device__ __forceinline__ void edge_weights(int nc, int ls, int i, int j, int l, Val val, Add add,
                                                      Scale scale, V* w) {
  auto C = [&](int p, int q, int r, int axis) { return val(coef_index<D>(nc, p >> ls, q >> ls, r >> ls, axis)); };
  if constexpr (D == 2) {
    // x edge from (p, q): cells (p, q), (p, q-1); y edge from (p, q): cells (p, q), (p-1, q)
    auto wx = [&](int p, int q) { return scale(add(C(p, q, 0, 0), C(p, q - 1, 0, 0))); };
    auto wy = [&](int p, int q) { return scale(add(C(p, q, 0, 1), C(p - 1, q, 0, 1))); };
    w[0] = wx(i - 1, j);
    w[1] = wx(i, j);
    w[2] = wy(i, j - 1);
    w[3] = wy(i, j);
  } else {
    auto tw = [&](V a, V b, V c, V d) { return scale(add(add(add(a, a), add(b, b)), add(c, d))); };
    auto wx = [&](int p, int q, int r) {
      return tw(C(p, q, r, 0), C(p, q - 1, r - 1, 0), C(p, q - 1, r, 0), C(p, q, r - 1, 0));
    };
    auto wy = [&](int p, int q, int r) {
      return tw(C(p, q, r, 1), C(p - 1, q, r - 1, 1), C(p - 1, q, r, 1), C(p, q, r - 1, 1));
    };
    auto wz = [&](int p, int q, int r) {
      return tw(C(p, q, r, 2), C(p - 1, q - 1, r, 2), C(p - 1, q, r, 2), C(p, q - 1, r, 2));
    };
    w[0] = wx(i - 1, j, l);
    w[1] = wx(i, j, l);
    w[2] = wy(i, j - 1, l);
    w[3] = wy(i, j, l);
    w[4] = wz(i, j, l - 1);
    w[5] = wz(i, j, l);
  }
}

// The edge weights in FP64 / FP32 (T = double reads a64, T = float reads a32).
template <int D, typename T>
__host__ __device__ __forceinline__ void edge_weights_t(const VarCoef& vc, int ls, int i, int j, int l, T* w) {
  const T* tab = nullptr;
  if constexpr (sizeof(T) == 8) tab = reinterpret_cast<const T*>(vc.a64);
  else tab = reinterpret_cast<const T*>(vc.a32);
  edge_weights<D, T>(
      vc.nc, ls, i, j, l, [&](int k) { return tab[k]; }, [](T x, T y) { return x + y; },
      [](T x) { return D == 2 ? x * T(0.5) : x / T(6); }, w);
}

// Nonlinearity a*f(u) and its derivative (Sec. 4 examples; monotone for a > 0).
template <typename T>
__device__ __forceinline__ void f_eval(int kind, T a, T u, T& F, T& Fp) {
  switch (kind) {
    case FMG_F_CUBIC: {
      T t = a * (u * u);
      F = t * u;
      Fp = T(3) * t;
      break;
    }
    case FMG_F_EXPM1: {
      T e = expm1(u);
      F = a * e;
      Fp = F + a;
      break;
    }
    case FMG_F_LINEAR:
      F = a * u;
      Fp = a;
      break;
    case FMG_F_SIGNED_POW32: {
      T r = sqrt(fabs(u));
      F = a * u * r;
      Fp = T(1.5) * a * r;
      break;
    }
    default: {  // FMG_F_NEG_EXP_NEG
      T e = exp(-u);
      F = -a * e;
      Fp = a * e;
      break;
    }
  }
}

template <typename T>
__device__ __forceinline__ T f_only(int kind, T a, T u) {
  switch (kind) {
    case FMG_F_CUBIC: return a * (u * u) * u;
    case FMG_F_EXPM1: return a * expm1(u);
    case FMG_F_LINEAR: return a * u;
    case FMG_F_SIGNED_POW32: return a * u * sqrt(fabs(u));
    default: return -a * exp(-u);
  }
}

// ---------------------------------------------------------------------------------------
// Launchers (host side), defined in fmg_stencil.cu / fmg_newton.cu.  All take the stream
// and return the launch error.
// ---------------------------------------------------------------------------------------

// red-black Gauss-Seidel half sweep of colour `colour` (0 red, 1 black) on level geometry g
template <typename T>
cudaError_t launch_rbgs(int dim, LevelGeo g, T* u, const T* b, int colour, cudaStream_t s,
                        const VarCoef* vc = nullptr);

// b_c = P^T (b_f - A_f u_f), u_c = 0 (coarse arrays of geometry gc, fine gf).  With d_c the
// coarse level's first Chebyshev step from zero is fused in: u_c = d_c = e0 b_c.
template <typename TF, typename TC>
cudaError_t launch_residual_restrict(int dim, LevelGeo gf, const TF* u_f, const TF* b_f, LevelGeo gc,
                                     TC* b_c, TC* u_c, cudaStream_t s, TC* d_c = nullptr, double e0 = 0.0,
                                     const VarCoef* vc = nullptr);

// mixed path: b32 = (float)(b - A u) in FP64, u32 = 0 (same level); with d32 the first
// Chebyshev step from zero is fused in: u32 = d32 = e0 b32
cudaError_t launch_residual_to_f32(int dim, LevelGeo g, const double* u, const double* b, float* r32,
                                   float* e32, cudaStream_t s, float* d32 = nullptr, double e0 = 0.0,
                                   const VarCoef* vc = nullptr);

// r = b - A u (FP64, same level)
cudaError_t launch_residual(int dim, LevelGeo g, const double* u, const double* b, double* r, cudaStream_t s,
                            const VarCoef* vc = nullptr);

// u_f += P e_c  (add = 1) or u_f = P e_c (add = 0)
template <typename TF, typename TC>
cudaError_t launch_prolong(int dim, LevelGeo gc, const TC* e_c, LevelGeo gf, TF* u_f, int add, cudaStream_t s);

// u += (double) e32 (mixed path update)
cudaError_t launch_add_f32(LevelGeo g, int dim, double* u, const float* e32, cudaStream_t s);

// b = w (g - a f(u)) at interior nodes, 0 on the boundary (eq. 3.4 with vertex quadrature)
cudaError_t launch_nonlinear_rhs(int dim, LevelGeo g, const double* u, const double* gn, double* b, int kind,
                                 double a, cudaStream_t s);

// copy nodal array (same level)
cudaError_t launch_copy(const double* src, double* dst, long long n, cudaStream_t s);

// FP32 V-cycle coarsest solve: e32 = (float)(Ainv (double) b32); FP64: e = Ainv b
cudaError_t launch_coarse_solve_f64(int dim, LevelGeo g1, const double* Ainv, const double* b, double* u,
                                    cudaStream_t s);
cudaError_t launch_coarse_solve_f32(int dim, LevelGeo g1, const double* Ainv, const float* b, float* u,
                                    cudaStream_t s);

// Chebyshev-Jacobi smoothing, the colour-free alternative smoother: step k of the three-term
// Chebyshev iteration on D^{-1} A over [lmax/4, lmax], lmax = 2, is
//   z = D^{-1}(b - A u),  d <- cd[k] d + cr[k] z  (cd[0] = 0),  u <- u + d.
constexpr int kMaxCheb = 16;
struct ChebCoef {
  double cd[kMaxCheb];
  double cr[kMaxCheb];
};
// Coefficients of steps 0..kMaxCheb-1 (host).
ChebCoef cheb_coefficients();
// One Chebyshev step on level geometry g: reads u (stencil), b and d (k > 0), writes uo and d.
// With ec (the next coarser level's correction) the step's iterate is u + P ec (the cycle's
// prolongation, fused into its first post-smoothing step).
template <typename T>
cudaError_t launch_cheb(int dim, LevelGeo g, const T* u, T* uo, T* d, const T* b, double cd, double cr, bool first,
                        cudaStream_t s, const T* ec = nullptr);
// Launch shape of the Chebyshev step kernel: threads per block along x and nodes per thread
// along the outer axis.  cheb_shape: the autotuned shape of this device and size if there
// is one, else the default rule; set_cheb_shape records a tuned one (process-wide).
struct ChebShape {
  int block;
  int strip;
};
ChebShape cheb_shape(int dim, int n, int elem_bytes);
bool cheb_shape_tuned(int dim, int n, int elem_bytes, ChebShape* out);
void set_cheb_shape(int dim, int n, int elem_bytes, ChebShape sh);
template <typename T>
cudaError_t launch_cheb_shaped(int dim, LevelGeo g, const T* u, T* uo, T* d, const T* b, double cd, double cr,
                               bool first, ChebShape sh, cudaStream_t s, const T* ec = nullptr);
// Last Chebyshev step of the mixed path's top-level FP32 cycle fused with u64 += correction.
cudaError_t launch_cheb_add64(int dim, LevelGeo g, const float* u, const float* d, const float* b, double* u64,
                              double cd, double cr, bool first, cudaStream_t s, bool u_ff = false);
template <typename T>
cudaError_t launch_copy_t(const T* src, T* dst, long long n, cudaStream_t s);

// The whole V-cycle on levels jtop..1 in one CTA with shared-memory level arrays (level j
// has n0 << (j-1) cells per side); u (in/out) and b are level jtop's nodal arrays.  cheb:
// NULL for red-black Gauss-Seidel smoothing, else Chebyshev-Jacobi steps (nu_pre / nu_post
// of them), which need two more arrays per level.
template <typename T>
size_t coarse_cycle_smem(int dim, int n0, int jtop, bool cheb);
// The V(nu_pre, nu_post) cycle on levels jtop..1 in one CTA.  Ainv32: FP32 copy of A_1^{-1}
// (required for T = float).  zero_start: u is zero on entry (not read).
template <typename T>
cudaError_t launch_coarse_cycle(int dim, int n0, int jtop, T* u, const T* b, int nu_pre, int nu_post,
                                const double* Ainv, const float* Ainv32, const ChebCoef* cheb, bool zero_start,
                                cudaStream_t s);
// dst = (float) src, n values
cudaError_t launch_to_f32(const double* src, float* dst, long long n, cudaStream_t s);

// level-1 setup: Ainv = A_1^{-1} (dense, N_1 x N_1) by Cholesky; flags on failure
cudaError_t launch_coarse_inverse(int dim, LevelGeo g1, double* Ainv, DevState* st, cudaStream_t s,
                                  const VarCoef* vc = nullptr);

// level-1 exact semilinear solve (Algorithm 3.2 step 1): Newton, dense, one CTA
// out_ff: u is written as float-float (the mixed solve's level data)
cudaError_t launch_level1_newton(int dim, LevelGeo g1, const double* gn, double* u, int kind, double a,
                                 double tol, int maxit, bool f32_factor, DevState* st, cudaStream_t s,
                                 bool out_ff = false, const VarCoef* vc = nullptr);

// Augmented problem on V_H + span{u~} (Algorithm 3.1 step 2, eq. 3.6): one cooperative
// persistent kernel: precompute, Newton iterations, final update u = alpha u~ + P_{H->k} c.
struct AugBuffers {
  double* partials;   // two buffers of [items][nvals] (the Newton iterations alternate), then two
                      // buffers of [cells][nvals] cell sums
  const double* Ainv; // A_H^{-1} (level-1 inverse; kept with the buffers of the system)
  double* cfin;       // the final coarse iterate c ((1/H + 1)^d nodal values) and alpha, for the
                      // separate update kernel of the largest levels
  size_t partial_items;
  int bpc;            // blocks per coarse cell of the cooperative launch (all co-resident)
  int nt;             // threads per block
  size_t smem;        // dynamic shared memory per block
  int sms;            // multiprocessors of the device
  const int* jtab;     // the mixed path's Jacobian gather table (launch_aug_jtab, once per context)
  long long bar_spins; // grid-barrier polls before a timeout (0: the default, 2^25)
  int bar_skip;        // failure-detection test hook: block that skips its first arrival (-1: none)
};
// Launch shape of the cooperative augmented kernel on one level: column-chunk length and
// blocks per coarse cell.  aug_shape gives the tuned one (set_aug_shape, process-wide; tuned =
// false: the rule only) within the launch's limits, else the rule of launch_augmented.
struct AugShape {
  int chunk;
  int bpc;
};
AugShape aug_shape(int dim, int coarse_cells, int level, bool jac_f32, const AugBuffers& ab, bool tuned = true);
void set_aug_shape(int dim, int coarse_cells, int level, bool mixed, AugShape sh);
bool aug_shape_tuned(int dim, int coarse_cells, int level, bool mixed, AugShape* out);
// Fills bpc/nt/smem/partial_items for this device (occupancy-based), outside any capture.
void aug_configure(int dim, int coarse_cells, bool mixed, AugBuffers* ab);
int aug_nvals(int dim);
// ints of the mixed path's Jacobian gather table, and the kernel that fills it
size_t aug_jtab_ints(int dim, int coarse_cells);
cudaError_t launch_aug_jtab(int dim, int coarse_cells, int* tab, cudaStream_t s);
// jac_f32: Jacobian moments in FP32 (residual stays FP64) -- the mixed-precision path.
// fixed_point: the fixed-point iteration on the Galerkin stiffness instead of Newton.
// cluster_size > 0: the thread-block-cluster variant (no cooperative launch; used when many
// instances run concurrently), with that many CTAs; 0: the cooperative grid variant.
// jac_f32 (mixed path): u and gn hold float-float values; out_f64: the result u is written as
// FP64 (the last correction step of a solve).
cudaError_t launch_augmented(int dim, int coarse_cells, int level, LevelGeo gk, double* u, const double* gn,
                             int kind, double a, double tol, int maxit, bool jac_f32, const AugBuffers& ab,
                             DevState* st, int level_index, cudaStream_t s, int cluster_size = 0, int fixed_point = 0,
                             int out_f64 = 0, const VarCoef* vc = nullptr);
// Largest usable cluster size (<= 16, <= number of coarse cells) for the cluster variant, 0 if none.
int aug_cluster_size(int dim, int coarse_cells, bool jac_f32, size_t smem);

// Float-float level data of the mixed solve (fmg_ff.cu): the level iterate u, the linear
// right-hand side b and g stored as float-float pairs in the 8-byte slots of the FP64 arrays.
// Residual r = b - A_k u into FP32 (with d32: the first Chebyshev step from zero, e = d = e0 r).
cudaError_t launch_residual_ff(int dim, LevelGeo g, const double* u_ff, const double* b_ff, float* r32, float* e32,
                               cudaStream_t s, float* d32 = nullptr, double e0 = 0.0, const VarCoef* vc = nullptr);
// b = w (g - a f(u)) (eq. 3.4, vertex rule)
cudaError_t launch_nonlinear_rhs_ff(int dim, LevelGeo g, const double* u_ff, const double* g_ff, double* b_ff,
                                    int kind, double a, cudaStream_t s);
// FMG interpolation u_f = P u_c on the interior fine nodes
cudaError_t launch_prolong_ff(int dim, LevelGeo gc, const double* uc_ff, LevelGeo gf, double* uf_ff, cudaStream_t s);
// u += e (FP32 correction)
cudaError_t launch_add_f32_ff(LevelGeo g, double* u_ff, const float* e32, cudaStream_t s);
// The start of level g in one pass: u = P u_c (FMG interpolation), b = w (g - a f(u)), and the
// first residual r32 = b - A u with e32 (and d32 with e0) as launch_residual_ff writes them.
cudaError_t launch_level_start_ff(int dim, LevelGeo gc, const double* uc_ff, LevelGeo g, double* u_ff,
                                  const double* g_ff, double* b_ff, int kind, double a, float* r32, float* e32,
                                  float* d32, double e0, cudaStream_t s, const VarCoef* vc = nullptr);
// every level's g (and its float-float copy gf, with ff) from the fine g, its boundary zeroed
cudaError_t launch_rhs_levels(int dim, int nlev, const LevelGeo* geo, double* const* g, double* const* gf, bool ff,
                              cudaStream_t s);
// conversions (in place allowed)
cudaError_t launch_ff_from_f64(const double* src, double* dst_ff, long long n, cudaStream_t s);
cudaError_t launch_ff_to_f64(const double* src_ff, double* dst, long long n, cudaStream_t s);

// Fused FP32 cycle kernels of the mixed path (fmg_fused.cu): 2D, nu in {1, 2}.
bool fused_cycle_supported(int dim, int nu_pre, int nu_post);
// nu sweeps from zero on level g, then b_c = P^T (b - A u), u_c = 0 on the next coarser level
cudaError_t launch_pre_fused(int dim, LevelGeo g, int nu, const float* b, float* u_out, float* bc, float* uc,
                             cudaStream_t s);
// u = u_in + P e_c, nu black-red sweeps; stored in u_out, or added to u64_top when non-NULL
cudaError_t launch_post_fused(int dim, LevelGeo g, int nu, const float* u_in, const float* ec, const float* b,
                              float* u_out, double* u64_top, cudaStream_t s, bool u_ff = false);

// Sets the calling thread's error message (what fmg_last_error(NULL) returns).
// Context services for the request server (fmg_capi.cu).
cudaStream_t ctx_stream(const fmg_ctx* c);
size_t ctx_bytes(const fmg_ctx* c);
size_t ctx_fine_nodes(const fmg_ctx* c);
// Switches the context to the cluster-variant Newton kernel, which any number of solves can
// run concurrently (drops a graph captured with the cooperative kernel).
fmg_status ctx_make_concurrent(fmg_ctx* c);
// Queues on the context stream: g from host, the solve graph, u and the DevState to host.
fmg_status ctx_enqueue(fmg_ctx* c, const double* g_host, double* u_host, DevState* state_host);
// Status and statistics of a finished solve from its DevState.
fmg_status ctx_decode(fmg_ctx* c, const DevState& h, fmg_stats* st);
const char* ctx_error(const fmg_ctx* c);

// Raises a kernel's dynamic shared-memory limit on the current device to at least `bytes`
// (never lowers it: contexts of different sizes share the kernels, and a graph captured
// for a larger one must keep launching after a smaller one was set up).
cudaError_t raise_dyn_smem(const void* kernel, size_t bytes);

void set_thread_error(const std::string& msg);

}  // namespace fmg

// Host side of the C ABI declared in include/fmg.h: the level hierarchy, the schedule of
// Algorithm 3.2 (full multigrid) and Algorithm 3.1 (one correction step), CUDA-graph capture
// of the whole solve, and the component operations.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "fmg_internal.cuh"
#include "fmg_phase.cuh"

using namespace fmg;

struct fmg_ctx {
  fmg_params p;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int nlev = 0;
  LevelGeo geo[kMaxLevels];
  double* u[kMaxLevels] = {};
  double* b[kMaxLevels] = {};
  double* g[kMaxLevels] = {};
  double* gf[kMaxLevels] = {};    // mixed path: g as float-float (the solve reads this copy)
  float* u32[kMaxLevels] = {};
  float* b32[kMaxLevels] = {};
  float* u32b[kMaxLevels] = {};   // second FP32 buffer: output of the fused pre-smoothing kernel,
                                  // or the Chebyshev smoother's second iterate (mixed path)
  float* d32[kMaxLevels] = {};    // Chebyshev step direction (mixed path)
  double* ua[kMaxLevels] = {};    // Chebyshev second iterate and direction (FP64 path and ops)
  double* dd[kMaxLevels] = {};
  ChebCoef cheb = {};
  double* Ainv = nullptr;
  float* Ainv32 = nullptr;   // FP32 copy of A_1^{-1} for the FP32 one-CTA cycles
  DevState* st = nullptr;
  AugBuffers ab = {};
  VarCoef vc = {};   // the coefficient A(x) on the device (vc.a64 == nullptr: A = I)
  void* arena = nullptr;
  size_t arena_bytes = 0;
  bool own_arena = false;
  bool own_stream = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  unsigned pending_flags = 0;
  int graph_kernels = 0;
  int cluster_aug = 0;   // > 0: cluster-variant Newton kernel of that size (batches, the server)
  // kernel timing (diagnostics): event pairs recorded inside the captured graph
  bool timing = false;
  struct Timed {
    int kind, level;
    cudaEvent_t e0, e1;
  };
  std::vector<Timed> timed;
  size_t timed_next = 0;
  std::string err;
};

struct fmg_batch {
  std::vector<fmg_ctx*> cs;
  cudaStream_t launch = nullptr;
  bool own_launch = false;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int mode = FMG_BATCH_BRANCHES;
  int kernels = 0;             // kernel nodes of the graph
  int groups = 0;              // phase groups (FMG_BATCH_PHASES)
};

namespace {

thread_local std::string t_err;

fmg_status fail(fmg_ctx* c, fmg_status s, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    t_err = msg;
  return s;
}

#define CK(ctx, expr)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail((ctx), FMG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));    \
  } while (0)

const char* validate(const fmg_params* p) {
  if (!p) return "params is NULL";
  if (p->dim != 2 && p->dim != 3) return "dim must be 2 or 3";
  if (p->coarse_cells < 2 || (p->coarse_cells & 1)) return "coarse_cells must be even and >= 2";
  if (p->dim == 2 && p->coarse_cells > 8) return "2D coarse_cells must be <= 8 (dense augmented system)";
  if (p->dim == 3 && p->coarse_cells > 4) return "3D coarse_cells must be <= 4 (dense augmented system)";
  if (p->refinements < 0 || p->refinements >= kMaxLevels - 1) return "refinements out of range";
  const long long nf = (long long)p->coarse_cells << p->refinements;
  if (p->dim == 2 && nf > 32768) return "2D fine mesh larger than 32768 cells per side";
  if (p->dim == 3 && nf > 1024) return "3D fine mesh larger than 1024 cells per side";
  if (p->f < 0 || p->f > 4) return "unknown nonlinearity";
  if (!(p->f_scale > 0.0) || !std::isfinite(p->f_scale)) return "f_scale must be finite and > 0";
  if (p->m_vcycles < 1 || p->m_vcycles > 64) return "m_vcycles must be in 1..64";
  if (p->nu_pre < 0 || p->nu_post < 0 || p->nu_pre > 64 || p->nu_post > 64) return "nu out of range";
  if (p->p_corrections < 1 || p->p_corrections > 64) return "p_corrections must be in 1..64";
  if (p->precision != FMG_PREC_FP64 && p->precision != FMG_PREC_MIXED) return "unknown precision";
  if (!(p->newton_tol > 0.0) || !(p->level1_tol > 0.0)) return "tolerances must be > 0";
  if (p->newton_maxit < 1 || p->newton_maxit > kMaxNewton) return "newton_maxit must be in 1..64";
  if (p->level1_maxit < 1 || p->level1_maxit > kMaxNewton) return "level1_maxit must be in 1..64";
  if (p->smoother != FMG_SMOOTHER_RBGS && p->smoother != FMG_SMOOTHER_CHEBYSHEV) return "unknown smoother";
  if (p->nonlinear != FMG_NONLINEAR_NEWTON && p->nonlinear != FMG_NONLINEAR_FIXED_POINT)
    return "unknown nonlinear solver";
  if (p->smoother == FMG_SMOOTHER_CHEBYSHEV && (p->nu_pre > kMaxCheb || p->nu_post > kMaxCheb))
    return "Chebyshev smoothing takes at most 16 steps";
  if (p->coefficient) {
    if (p->smoother != FMG_SMOOTHER_RBGS) return "a variable coefficient takes the red-black smoother";
    const long long n = ipow(p->coarse_cells, p->dim) * p->dim;
    for (long long i = 0; i < n; ++i)
      if (!(p->coefficient[i] > 0.0) || !std::isfinite(p->coefficient[i]))
        return "coefficient entries must be finite and > 0";
  }
  return nullptr;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Lays out (or only sizes, when base == nullptr) every device array of a context.
size_t layout(fmg_ctx* c, const fmg_params* p, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* r = base ? base + off : nullptr;
    off += align_up(bytes);
    return r;
  };
  const int nlev = p->refinements + 1;
  for (int k = 0; k < nlev; ++k) {
    const int n = p->coarse_cells << k;
    const long long nodes = ipow(n + 1, p->dim);
    if (c) {
      c->geo[k].n = n;
      c->geo[k].np = n + 1;
      c->geo[k].nodes = nodes;
    }
    double* u = (double*)take(nodes * 8);
    double* b = (double*)take(nodes * 8);
    double* g = (double*)take(nodes * 8);
    float* u32 = nullptr;
    float* b32 = nullptr;
    float* u32b = nullptr;
    float* d32 = nullptr;
    double* ua = nullptr;
    double* dd = nullptr;
    double* gf = nullptr;
    const bool cheb = p->smoother == FMG_SMOOTHER_CHEBYSHEV;
    if (p->precision == FMG_PREC_MIXED) {
      gf = (double*)take(nodes * 8);
      u32 = (float*)take(nodes * 4);
      b32 = (float*)take(nodes * 4);
      if (cheb || fused_cycle_supported(p->dim, p->nu_pre, p->nu_post)) u32b = (float*)take(nodes * 4);
      if (cheb) d32 = (float*)take(nodes * 4);
    }
    if (cheb) {
      ua = (double*)take(nodes * 8);
      dd = (double*)take(nodes * 8);
    }
    if (c && base) {
      c->u[k] = u;
      c->b[k] = b;
      c->g[k] = g;
      c->gf[k] = gf;
      c->u32[k] = u32;
      c->b32[k] = b32;
      c->u32b[k] = u32b;
      c->d32[k] = d32;
      c->ua[k] = ua;
      c->dd[k] = dd;
    }
  }
  const int m = p->coarse_cells - 1;
  const long long N1 = ipow(m, p->dim);
  double* Ainv = (double*)take(N1 * N1 * 8);
  float* Ainv32 = (float*)take(N1 * N1 * 4);
  DevState* st = (DevState*)take(sizeof(DevState));
  AugBuffers cfg = {};
  aug_configure(p->dim, p->coarse_cells, p->precision == FMG_PREC_MIXED, &cfg);
  const size_t items = cfg.partial_items;
  double* partials = (double*)take(2 * (items + ipow(p->coarse_cells, p->dim)) * aug_nvals(p->dim) * 8);
  double* cfin = (double*)take((ipow(p->coarse_cells + 1, p->dim) + 1) * 8);
  int* jtab = (int*)take(aug_jtab_ints(p->dim, p->coarse_cells) * 4);
  // the coefficient table in FP64, FP32 and float-float (a row of d entries per cell of T_H)
  const long long ncoef = ipow(p->coarse_cells, p->dim) * p->dim;
  double* a64 = (double*)take(ncoef * 8);
  float* a32 = (float*)take(ncoef * 4);
  double* aff = (double*)take(ncoef * 8);
  if (c && base) {
    c->vc.a64 = p->coefficient ? a64 : nullptr;
    c->vc.a32 = p->coefficient ? a32 : nullptr;
    c->vc.aff = p->coefficient ? aff : nullptr;
    c->vc.nc = p->coarse_cells;
    c->Ainv = Ainv;
    c->Ainv32 = Ainv32;
    c->st = st;
    c->ab = cfg;
    c->ab.partials = partials;
    c->ab.Ainv = Ainv;
    c->ab.cfin = cfin;
    c->ab.jtab = jtab;
    c->ab.bar_spins = 0;
    c->ab.bar_skip = -1;
  }
  return off;
}

// ------------------------------------------------------------------ kernel timing
// In timing mode every instrumented launch is bracketed by two events recorded on the
// context stream; inside a capture they become event-record nodes of the graph, so each
// replay refreshes the timestamps.  Events are created on the first capture and reused.
// tbegin allocates a slot (or returns -1 when timing is off) and records its first event;
// tend records the second event of that slot.  Slots nest freely.
cudaError_t tbegin(fmg_ctx* c, int kind, int level, int* slot) {
  *slot = -1;
  if (!c->timing) return cudaSuccess;
  cudaError_t e;
  if (c->timed_next == c->timed.size()) {
    fmg_ctx::Timed t{kind, level, nullptr, nullptr};
    if ((e = cudaEventCreate(&t.e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&t.e1)) != cudaSuccess) {
      cudaEventDestroy(t.e0);
      return e;
    }
    c->timed.push_back(t);
  }
  const size_t i = c->timed_next++;
  c->timed[i].kind = kind;
  c->timed[i].level = level;
  *slot = (int)i;
  return cudaEventRecordWithFlags(c->timed[i].e0, c->stream, cudaEventRecordExternal);
}

cudaError_t tend(fmg_ctx* c, int slot) {
  if (slot < 0 || (size_t)slot >= c->timed.size()) return cudaSuccess;
  return cudaEventRecordWithFlags(c->timed[slot].e1, c->stream, cudaEventRecordExternal);
}

// The schedule's launch calls: on failure the innermost call's text is kept (per thread) so
// that a capture error can name the launch that failed.
thread_local const char* t_site = nullptr;
#define TRY(...)                                  \
  do {                                            \
    cudaError_t e_ = (__VA_ARGS__);               \
    if (e_ != cudaSuccess) {                      \
      if (!t_site) t_site = #__VA_ARGS__;         \
      return e_;                                  \
    }                                             \
  } while (0)

// ------------------------------------------------------------------ schedule pieces
const ChebCoef* cheb_coef(const fmg_ctx* c) {
  return c->p.smoother == FMG_SMOOTHER_CHEBYSHEV ? &c->cheb : nullptr;
}

// Chebyshev-Jacobi steps first..steps-1 on A u = b at level j (one stencil pass each, d the
// step direction), the iterate starting in `cur` and alternating with `oth`; *end receives
// the buffer that holds the result.  ec: the coarse correction, prolongated into the first
// step's iterate (the cycle's prolongation fused into its first post-smoothing step).
template <typename T>
cudaError_t cheb_run(fmg_ctx* c, int j, T* cur, T* oth, T* d, const T* b, int first, int steps, bool top, T** end,
                     const T* ec = nullptr) {
  const LevelGeo g = c->geo[j - 1];
  for (int k = first; k < steps; ++k) {
    int slot = -1;
    if (top) TRY(tbegin(c, FMG_KT_SMOOTH_TOP, j, &slot));
    TRY(launch_cheb<T>(c->p.dim, g, cur, oth, d, b, c->cheb.cd[k], c->cheb.cr[k], k == 0, c->stream,
                       k == first ? ec : nullptr));
    TRY(tend(c, slot));
    T* t = cur;
    cur = oth;
    oth = t;
  }
  *end = cur;
  return cudaSuccess;
}

// The buffer that a Chebyshev step 0 taken from a zero start (fused into the kernel that
// produces b) writes, so that the remaining steps first..steps-1 end in u: u when their
// number is even, alt when it is odd.
template <typename T>
T* cheb_start(T* u, T* alt, int steps) {
  return ((steps - 1) & 1) ? alt : u;
}

// Chebyshev-Jacobi steps first..steps-1 on A u = b at level j; the iterate starts in
// cheb_start(u, alt, steps) when first = 1 (step 0 fused upstream), in u otherwise, and the
// result ends in u (a copy only when first = 0 and the step count is odd).
template <typename T>
cudaError_t cheb_steps(fmg_ctx* c, int j, T* u, T* alt, T* d, const T* b, int steps, bool top, int first = 0,
                       const T* ec = nullptr) {
  T* start = first ? cheb_start(u, alt, steps) : u;
  T* end = nullptr;
  TRY(cheb_run<T>(c, j, start, start == u ? alt : u, d, b, first, steps, top, &end, ec));
  if (end != u) TRY(launch_copy_t<T>(end, u, c->geo[j - 1].nodes, c->stream));
  return cudaSuccess;
}

// The coefficient for the launch calls: nullptr when A = I (the constant-coefficient kernels).
const VarCoef* vcp(const fmg_ctx* c) { return c->vc.a64 ? &c->vc : nullptr; }

// Largest level handled by the one-CTA coarse cycle: its level arrays (u and b of every level
// up to it) must fit in shared memory; 2D up to 64 cells per side, 3D up to 16.  With a
// variable coefficient every level above 1 runs the per-level kernels.
template <typename T>
int coarse_cycle_top(const fmg_ctx* c) {
  if (c->vc.a64) return 1;
  const int nmax = c->p.dim == 2 ? 64 : 16;
  int j = 1;
  while (j < c->nlev && c->geo[j].n <= nmax &&
         coarse_cycle_smem<T>(c->p.dim, c->p.coarse_cells, j + 1, c->p.smoother == FMG_SMOOTHER_CHEBYSHEV) <= 200 * 1024)
    ++j;
  return j;
}

// Factor of Chebyshev step 0 from a zero start at level j: u = d = cr_0 D^{-1} b.
double cheb_e0(const fmg_ctx* c, int j) {
  const double bscale = c->p.dim == 2 ? 1.0 : (double)c->geo[j - 1].n;
  return c->cheb.cr[0] * bscale / (2.0 * c->p.dim);
}

// Whether a coarse level j, entered from zero by the restriction, takes its first Chebyshev
// step inside that restriction (it runs the per-level kernels and pre-smooths at all).
template <typename T>
bool fuse_first_step(const fmg_ctx* c, int j) {
  return c->p.smoother == FMG_SMOOTHER_CHEBYSHEV && c->p.nu_pre >= 1 && j > coarse_cycle_top<T>(c);
}

// Whether the mixed cycle on level k runs the fused 2D FP32 kernels (red-black smoothing with
// the constant-coefficient stencil; their buffers exist).
bool fused_cycle_used(const fmg_ctx* c, int k) {
  return c->u32b[k - 1] && c->p.smoother == FMG_SMOOTHER_RBGS && !c->vc.a64;
}

cudaError_t vcycle(fmg_ctx* c, int j, double* u, const double* b, bool top = false, bool started = false) {
  const int dim = c->p.dim;
  cudaStream_t s = c->stream;
  if (j == 1) {
    TRY(launch_coarse_solve_f64(dim, c->geo[0], c->Ainv, b, u, s));
    return cudaSuccess;
  }
  if (j <= coarse_cycle_top<double>(c)) {
    // below the top level the restriction has zeroed u
    TRY(launch_coarse_cycle<double>(dim, c->p.coarse_cells, j, u, b, c->p.nu_pre, c->p.nu_post, c->Ainv, nullptr,
                                    cheb_coef(c), !top, s));
    return cudaSuccess;
  }
  const LevelGeo gf = c->geo[j - 1], gc = c->geo[j - 2];
  const bool cheb = c->p.smoother == FMG_SMOOTHER_CHEBYSHEV;
  if (cheb) TRY(cheb_steps<double>(c, j, u, c->ua[j - 1], c->dd[j - 1], b, c->p.nu_pre, top, started ? 1 : 0));
  for (int it = 0; !cheb && it < c->p.nu_pre; ++it) {
    int slot = -1;
    if (top) TRY(tbegin(c, FMG_KT_SMOOTH_TOP, j, &slot));
    TRY(launch_rbgs<double>(dim, gf, u, b, 0, s, vcp(c)));
    TRY(launch_rbgs<double>(dim, gf, u, b, 1, s, vcp(c)));
    TRY(tend(c, slot));
  }
  const bool fuse = fuse_first_step<double>(c, j - 1);
  double* uc0 = fuse ? cheb_start(c->u[j - 2], c->ua[j - 2], c->p.nu_pre) : c->u[j - 2];
  TRY(launch_residual_restrict<double, double>(dim, gf, u, b, gc, c->b[j - 2], uc0, s,
                                               fuse ? c->dd[j - 2] : nullptr, fuse ? cheb_e0(c, j - 1) : 0.0, vcp(c)));
  TRY(vcycle(c, j - 1, c->u[j - 2], c->b[j - 2], false, fuse));
  TRY(launch_prolong<double, double>(dim, gc, c->u[j - 2], gf, u, 1, s));
  if (cheb) TRY(cheb_steps<double>(c, j, u, c->ua[j - 1], c->dd[j - 1], b, c->p.nu_post, top));
  for (int it = 0; !cheb && it < c->p.nu_post; ++it) {
    int slot = -1;
    if (top) TRY(tbegin(c, FMG_KT_SMOOTH_TOP, j, &slot));
    TRY(launch_rbgs<double>(dim, gf, u, b, 1, s, vcp(c)));
    TRY(launch_rbgs<double>(dim, gf, u, b, 0, s, vcp(c)));
    TRY(tend(c, slot));
  }
  return cudaSuccess;
}

// FP32 cycle below level j with the fused kernels: the correction starts at zero on every
// level (the parent's restriction zeroes it; the top level's defect equation starts at zero),
// pre-smoothing writes the level's second buffer, post-smoothing reads it back into the first
// one -- or, on the top level, adds the result to the iterate u64 (FP64 in the ops, float-float
// in a mixed solve: top_ff).
cudaError_t vcycle32_fused(fmg_ctx* c, int j, double* u64_top, bool top_ff = false) {
  const int dim = c->p.dim;
  cudaStream_t s = c->stream;
  if (j == 1) {
    TRY(launch_coarse_solve_f32(dim, c->geo[0], c->Ainv, c->b32[0], c->u32[0], s));
    return cudaSuccess;
  }
  if (j <= coarse_cycle_top<float>(c)) {
    // the FP32 cycles solve for a correction from zero on every level
    TRY(launch_coarse_cycle<float>(dim, c->p.coarse_cells, j, c->u32[j - 1], c->b32[j - 1], c->p.nu_pre,
                                   c->p.nu_post, c->Ainv, c->Ainv32, cheb_coef(c), true, s));
    if (u64_top && top_ff) TRY(launch_add_f32_ff(c->geo[j - 1], u64_top, c->u32[j - 1], s));
    if (u64_top && !top_ff) TRY(launch_add_f32(c->geo[j - 1], dim, u64_top, c->u32[j - 1], s));
    return cudaSuccess;
  }
  const LevelGeo gf = c->geo[j - 1];
  int slot = -1;
  if (u64_top) TRY(tbegin(c, FMG_KT_PRE_TOP, j, &slot));
  TRY(launch_pre_fused(dim, gf, c->p.nu_pre, c->b32[j - 1], c->u32b[j - 1], c->b32[j - 2], c->u32[j - 2], s));
  TRY(tend(c, slot));
  TRY(vcycle32_fused(c, j - 1, nullptr));
  slot = -1;
  if (u64_top) TRY(tbegin(c, FMG_KT_POST_TOP, j, &slot));
  TRY(launch_post_fused(dim, gf, c->p.nu_post, c->u32b[j - 1], c->u32[j - 2], c->b32[j - 1], c->u32[j - 1], u64_top,
                        s, top_ff));
  return tend(c, slot);
}

// FP32 cycle on level j (unfused kernels).  started: Chebyshev step 0 was already taken by the
// kernel that produced b; u64_top (top level of the mixed path): the last post-smoothing step
// is fused with the update u64 += correction (u64 FP64, or float-float when top_ff).
cudaError_t vcycle32(fmg_ctx* c, int j, bool top = false, bool started = false, double* u64_top = nullptr,
                     bool top_ff = false) {
  const int dim = c->p.dim;
  cudaStream_t s = c->stream;
  float* u = c->u32[j - 1];
  const float* b = c->b32[j - 1];
  if (j == 1) {
    TRY(launch_coarse_solve_f32(dim, c->geo[0], c->Ainv, b, u, s));
    return cudaSuccess;
  }
  if (j <= coarse_cycle_top<float>(c)) {
    TRY(launch_coarse_cycle<float>(dim, c->p.coarse_cells, j, u, b, c->p.nu_pre, c->p.nu_post, c->Ainv, c->Ainv32,
                                   cheb_coef(c), true, s));
    return cudaSuccess;
  }
  const LevelGeo gf = c->geo[j - 1], gc = c->geo[j - 2];
  const bool cheb = c->p.smoother == FMG_SMOOTHER_CHEBYSHEV;
  if (cheb) TRY(cheb_steps<float>(c, j, u, c->u32b[j - 1], c->d32[j - 1], b, c->p.nu_pre, top, started ? 1 : 0));
  for (int it = 0; !cheb && it < c->p.nu_pre; ++it) {
    int slot = -1;
    if (top) TRY(tbegin(c, FMG_KT_SMOOTH_TOP, j, &slot));
    TRY(launch_rbgs<float>(dim, gf, u, b, 0, s, vcp(c)));
    TRY(launch_rbgs<float>(dim, gf, u, b, 1, s, vcp(c)));
    TRY(tend(c, slot));
  }
  const bool fuse = fuse_first_step<float>(c, j - 1);
  float* uc0 = fuse ? cheb_start(c->u32[j - 2], c->u32b[j - 2], c->p.nu_pre) : c->u32[j - 2];
  TRY(launch_residual_restrict<float, float>(dim, gf, u, b, gc, c->b32[j - 2], uc0, s,
                                             fuse ? c->d32[j - 2] : nullptr, fuse ? cheb_e0(c, j - 1) : 0.0, vcp(c)));
  TRY(vcycle32(c, j - 1, false, fuse));
  // the prolongation u += P e_c, fused into the first post-smoothing Chebyshev step when that
  // is a plain step (not the top level's single step fused with the update)
  const bool prol_fused = cheb && c->p.nu_post >= 1 && (!u64_top || c->p.nu_post >= 2);
  const float* ec = prol_fused ? c->u32[j - 2] : nullptr;
  if (!prol_fused) TRY(launch_prolong<float, float>(dim, gc, c->u32[j - 2], gf, u, 1, s));
  if (cheb && u64_top && c->p.nu_post >= 1) {
    // steps 0..last-1, then the last one fused with the update of u64, reading whichever
    // buffer holds the iterate
    const int last = c->p.nu_post - 1;
    float* end = nullptr;
    TRY(cheb_run<float>(c, j, u, c->u32b[j - 1], c->d32[j - 1], b, 0, last, top, &end, ec));
    TRY(launch_cheb_add64(dim, gf, end, c->d32[j - 1], b, u64_top, c->cheb.cd[last], c->cheb.cr[last], last == 0,
                          s, top_ff));
    return cudaSuccess;
  }
  if (cheb) TRY(cheb_steps<float>(c, j, u, c->u32b[j - 1], c->d32[j - 1], b, c->p.nu_post, top, 0, ec));
  for (int it = 0; !cheb && it < c->p.nu_post; ++it) {
    int slot = -1;
    if (top) TRY(tbegin(c, FMG_KT_SMOOTH_TOP, j, &slot));
    TRY(launch_rbgs<float>(dim, gf, u, b, 1, s, vcp(c)));
    TRY(launch_rbgs<float>(dim, gf, u, b, 0, s, vcp(c)));
    TRY(tend(c, slot));
  }
  if (u64_top && top_ff) TRY(launch_add_f32_ff(gf, u64_top, u, s));
  if (u64_top && !top_ff) TRY(launch_add_f32(gf, dim, u64_top, u, s));
  return cudaSuccess;
}

// One multigrid cycle for A_k u = b at the top level k, in the context's precision.
cudaError_t top_cycle(fmg_ctx* c, int k, double* u, const double* b) {
  if (c->p.precision == FMG_PREC_FP64 || k == 1) return vcycle(c, k, u, b, true);
  const LevelGeo g = c->geo[k - 1];
  // defect correction: FP64 residual -> FP32 cycle from e = 0 -> FP64 update (with Chebyshev
  // smoothing the cycle's first step is fused into the residual and its last into the update)
  const bool fuse = fuse_first_step<float>(c, k);
  float* e0buf = fuse ? cheb_start(c->u32[k - 1], c->u32b[k - 1], c->p.nu_pre) : c->u32[k - 1];
  TRY(launch_residual_to_f32(c->p.dim, g, u, b, c->b32[k - 1], e0buf, c->stream,
                             fuse ? c->d32[k - 1] : nullptr, fuse ? cheb_e0(c, k) : 0.0, vcp(c)));
  if (fused_cycle_used(c, k)) return vcycle32_fused(c, k, u);
  if (k > coarse_cycle_top<float>(c)) return vcycle32(c, k, true, fuse, u);
  TRY(vcycle32(c, k, true));
  TRY(launch_add_f32(g, c->p.dim, u, c->u32[k - 1], c->stream));
  return cudaSuccess;
}

// The same cycle on the mixed solve's float-float level data: float-float residual -> FP32
// cycle from e = 0 -> float-float update (the residual and the update in FP32 error-free
// transformations instead of FP64 arithmetic).
// residual_ready: the residual (and the first step from zero) is already in b32 / u32 (the
// level start computed it).
cudaError_t top_cycle_ff(fmg_ctx* c, int k, double* u, const double* b, bool residual_ready = false) {
  const LevelGeo g = c->geo[k - 1];
  const bool fuse = fuse_first_step<float>(c, k);
  float* e0buf = fuse ? cheb_start(c->u32[k - 1], c->u32b[k - 1], c->p.nu_pre) : c->u32[k - 1];
  if (!residual_ready)
    TRY(launch_residual_ff(c->p.dim, g, u, b, c->b32[k - 1], e0buf, c->stream, fuse ? c->d32[k - 1] : nullptr,
                           fuse ? cheb_e0(c, k) : 0.0, vcp(c)));
  if (fused_cycle_used(c, k)) return vcycle32_fused(c, k, u, true);
  if (k > coarse_cycle_top<float>(c)) return vcycle32(c, k, true, fuse, u, true);
  TRY(vcycle32(c, k, true));
  TRY(launch_add_f32_ff(g, u, c->u32[k - 1], c->stream));
  return cudaSuccess;
}

// Algorithm 3.1 at level k >= 2 on the level-k array u (FP64 contexts).
cudaError_t correction_step(fmg_ctx* c, int k, double* u) {
  if (c->p.precision == FMG_PREC_MIXED) return cudaErrorInvalidValue;
  const LevelGeo g = c->geo[k - 1];
  int slot_step = -1, slot_aug = -1;
  TRY(tbegin(c, FMG_KT_CORRECTION, k, &slot_step));
  // step 1: b = (g, v) - (f(x, u^{(l)}), v)   (eq. 3.4)
  TRY(launch_nonlinear_rhs(c->p.dim, g, u, c->g[k - 1], c->b[k - 1], c->p.f, c->p.f_scale, c->stream));
  for (int i = 0; i < c->p.m_vcycles; ++i) TRY(top_cycle(c, k, u, c->b[k - 1]));
  // step 2: semilinear problem on V_H + span{u~}  (eq. 3.6)
  TRY(tbegin(c, FMG_KT_AUGMENTED, k, &slot_aug));
  TRY(launch_augmented(c->p.dim, c->p.coarse_cells, k, g, u, c->g[k - 1], c->p.f, c->p.f_scale, c->p.newton_tol,
                       c->p.newton_maxit, c->p.precision == FMG_PREC_MIXED, c->ab, c->st, k - 1, c->stream,
                       c->cluster_aug, c->p.nonlinear == FMG_NONLINEAR_FIXED_POINT ? 1 : 0, 0, vcp(c)));
  TRY(tend(c, slot_aug));
  return tend(c, slot_step);
}

// Algorithm 3.1 at level k >= 2 on the mixed solve's float-float level data (u = u[k-1],
// b = b[k-1], g = gf[k-1]); out_f64: the result is left as FP64 (the solve's last step);
// from_coarse: u starts as the FMG interpolation of level k-1 (the first step of the level),
// formed here together with b and the first residual in one pass.
cudaError_t correction_step_ff(fmg_ctx* c, int k, bool out_f64, bool from_coarse = false) {
  const LevelGeo g = c->geo[k - 1];
  double* u = c->u[k - 1];
  int slot_step = -1, slot_aug = -1;
  TRY(tbegin(c, FMG_KT_CORRECTION, k, &slot_step));
  // step 1: b = (g, v) - (f(x, u^{(l)}), v)   (eq. 3.4)
  if (from_coarse) {
    const bool fuse = fuse_first_step<float>(c, k);
    float* e0buf = fuse ? cheb_start(c->u32[k - 1], c->u32b[k - 1], c->p.nu_pre) : c->u32[k - 1];
    TRY(launch_level_start_ff(c->p.dim, c->geo[k - 2], c->u[k - 2], g, u, c->gf[k - 1], c->b[k - 1], c->p.f,
                              c->p.f_scale, c->b32[k - 1], e0buf, fuse ? c->d32[k - 1] : nullptr,
                              fuse ? cheb_e0(c, k) : 0.0, c->stream, vcp(c)));
  } else {
    TRY(launch_nonlinear_rhs_ff(c->p.dim, g, u, c->gf[k - 1], c->b[k - 1], c->p.f, c->p.f_scale, c->stream));
  }
  for (int i = 0; i < c->p.m_vcycles; ++i) TRY(top_cycle_ff(c, k, u, c->b[k - 1], from_coarse && i == 0));
  // step 2: semilinear problem on V_H + span{u~}  (eq. 3.6)
  TRY(tbegin(c, FMG_KT_AUGMENTED, k, &slot_aug));
  TRY(launch_augmented(c->p.dim, c->p.coarse_cells, k, g, u, c->gf[k - 1], c->p.f, c->p.f_scale, c->p.newton_tol,
                       c->p.newton_maxit, true, c->ab, c->st, k - 1, c->stream, c->cluster_aug,
                       c->p.nonlinear == FMG_NONLINEAR_FIXED_POINT ? 1 : 0, out_f64 ? 1 : 0, vcp(c)));
  TRY(tend(c, slot_aug));
  return tend(c, slot_step);
}

cudaError_t run_fmg(fmg_ctx* c) {
  // programmatic serialization only for a context that runs alone (no cluster Newton kernel)
  PdlScope pdl(c->cluster_aug == 0);
  c->timed_next = 0;
  // per-solve statistics start at zero (flags, iteration counts, alphas)
  TRY(cudaMemsetAsync(c->st, 0, offsetof(DevState, alpha_cur), c->stream));
  // the mixed path keeps its level data as float-float; its last step leaves the FP64 result
  const bool mixed = c->p.precision == FMG_PREC_MIXED;
  TRY(launch_level1_newton(c->p.dim, c->geo[0], c->g[0], c->u[0], c->p.f, c->p.f_scale, c->p.level1_tol,
                           c->p.level1_maxit, mixed, c->st, c->stream, mixed && c->nlev > 1, vcp(c)));
  for (int k = 2; k <= c->nlev; ++k) {
    // u^{(0)}_{h_k} = u_{h_{k-1}}: the natural inclusion (the mixed path forms it in the pass
    // that starts its first correction step)
    if (!mixed)
      TRY(launch_prolong<double, double>(c->p.dim, c->geo[k - 2], c->u[k - 2], c->geo[k - 1], c->u[k - 1], 0,
                                         c->stream));
    for (int l = 0; l < c->p.p_corrections; ++l) {
      if (mixed)
        TRY(correction_step_ff(c, k, k == c->nlev && l == c->p.p_corrections - 1, l == 0));
      else
        TRY(correction_step(c, k, c->u[k - 1]));
    }
  }
  return cudaSuccess;
}

// Statistics and status of one solve from a host copy of its DevState.
fmg_status decode_state(fmg_ctx* c, const DevState& h, unsigned extra_flags, fmg_stats* st) {
  const unsigned flags = h.flags | extra_flags;
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->levels = c->nlev;
    st->level1_iters = h.level1_iters;
    for (int k = 0; k < 32 && k < kMaxLevels; ++k) {
      st->newton_iters[k] = h.newton_iters[k];
      st->alpha[k] = h.alpha[k];
    }
    st->flags = flags;
  }
  if (flags & kFlagTimeout) return fail(c, FMG_ERR_TIMEOUT, "a bounded device wait timed out");
  if (flags & kFlagNonfinite) return fail(c, FMG_ERR_NONFINITE, "non-finite value in an iterate");
  if (flags & (kFlagNewtonCap | kFlagNotSPD))
    return fail(c, FMG_ERR_NO_CONVERGENCE, "a Newton iteration hit its cap or met a non-SPD matrix");
  return FMG_OK;
}

fmg_status read_state(fmg_ctx* c, fmg_stats* st, bool accumulate_pending) {
  DevState h;
  CK(c, cudaStreamSynchronize(c->stream));
  CK(c, cudaMemcpy(&h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  const unsigned extra = accumulate_pending ? c->pending_flags : 0u;
  c->pending_flags = 0;
  return decode_state(c, h, extra, st);
}

fmg_status load_rhs(fmg_ctx* c, const double* g_fine, int on_device) {
  if (!g_fine) return fail(c, FMG_ERR_INVALID, "g is NULL");
  const int top = c->nlev - 1;
  CK(c, cudaMemcpyAsync(c->g[top], g_fine, c->geo[top].nodes * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  // the boundary ring, every coarser level by injection and the float-float copies: one launch
  CK(c, launch_rhs_levels(c->p.dim, c->nlev, c->geo, c->g, c->gf, c->p.precision == FMG_PREC_MIXED, c->stream));
  return FMG_OK;
}

fmg_status check_level(fmg_ctx* c, int level, int lo) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  if (level < lo || level > c->nlev) return fail(c, FMG_ERR_INVALID, "level out of range");
  return FMG_OK;
}

// Kernel nodes of a graph (the launches of one replay).
int graph_kernel_nodes(cudaGraph_t graph) {
  size_t nn = 0;
  int k = 0;
  if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
      }
  }
  return k;
}

// Captures the whole schedule of Algorithm 3.2 into the context's graph (once).
fmg_status ensure_graph(fmg_ctx* c) {
  if (c->gexec) return FMG_OK;
  {
    t_site = nullptr;
    CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = run_fmg(c);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(c, FMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2) +
                                       (t_site ? std::string(" at ") + t_site : std::string()));
    }
    c->graph_kernels = graph_kernel_nodes(graph);
    e = cudaGraphInstantiate(&c->gexec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      c->gexec = nullptr;
      return fail(c, FMG_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    c->graph = graph;
  }
  return FMG_OK;
}

// ------------------------------------------------------------------ phase-batched graph
// Phase groups per set of instances whose schedules agree, when the caller leaves it open.
constexpr int kDefaultPhaseSplit = 8;

// One step of an instance's captured schedule: a kernel launch (its phase-batchable form and
// its arguments packed as a table entry) or a memset.
struct PhaseStep {
  bool memset = false;
  cudaMemsetParams ms = {};
  const PhaseKernel* pk = nullptr;
  dim3 grid, block;
  unsigned smem = 0;
  dim3 cluster = dim3(0, 0, 0);   // x == 0: no cluster
  std::vector<unsigned char> args;
};

const std::vector<PhaseKernel>& phase_registry() {
  static const std::vector<PhaseKernel> reg = [] {
    std::vector<PhaseKernel> r;
    phase_kernels_stencil(r);
    phase_kernels_ff(r);
    phase_kernels_fused(r);
    phase_kernels_newton(r);
    return r;
  }();
  return reg;
}

const PhaseKernel* phase_lookup(const void* f) {
  for (const PhaseKernel& k : phase_registry())
    if (k.solo == f) return &k;
  return nullptr;
}

bool same_step(const PhaseStep& a, const PhaseStep& b) {
  if (a.memset != b.memset) return false;
  if (a.memset) return true;
  return a.pk == b.pk && a.grid.x == b.grid.x && a.grid.y == b.grid.y && a.block.x == b.block.x &&
         a.block.y == b.block.y && a.block.z == b.block.z && a.smem == b.smem && a.cluster.x == b.cluster.x &&
         a.cluster.y == b.cluster.y && a.cluster.z == b.cluster.z;
}

// Captures instance c's whole schedule (the cluster Newton kernel of size csz) on stream cap and
// reads it back as a chain of steps.  False, with the reason, if a node is neither a memset nor
// a phase-batchable kernel with a z extent of one.
bool phase_chain(fmg_ctx* c, int csz, cudaStream_t cap, std::vector<PhaseStep>& chain, std::string& why) {
  cudaStream_t saved = c->stream;
  const bool timing = c->timing;
  const int cluster = c->cluster_aug;
  c->stream = cap;
  c->cluster_aug = csz;
  c->timing = false;
  t_site = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  cudaError_t ce = e == cudaSuccess ? run_fmg(c) : e;
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) e = cudaStreamEndCapture(cap, &g);
  c->stream = saved;
  c->cluster_aug = cluster;
  c->timing = timing;
  if (ce != cudaSuccess || e != cudaSuccess) {
    why = std::string("capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : e);
    if (g) cudaGraphDestroy(g);
    return false;
  }
  bool ok = true;
  size_t nr = 0;
  cudaGraphNode_t node = nullptr;
  if (cudaGraphGetRootNodes(g, nullptr, &nr) != cudaSuccess || nr != 1 ||
      cudaGraphGetRootNodes(g, &node, &nr) != cudaSuccess) {
    why = "the schedule is not a single chain";
    ok = false;
  }
  while (ok && node) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(node, &t) != cudaSuccess) {
      why = "node type";
      ok = false;
      break;
    }
    if (t == cudaGraphNodeTypeKernel) {
      cudaKernelNodeParams kp = {};
      PhaseStep st;
      if (cudaGraphKernelNodeGetParams(node, &kp) != cudaSuccess || !(st.pk = phase_lookup(kp.func))) {
        why = "a kernel of the schedule has no phase-batched form";
        ok = false;
        break;
      }
      if (kp.gridDim.z != 1) {
        why = "a kernel of the schedule tiles z";
        ok = false;
        break;
      }
      st.grid = kp.gridDim;
      st.block = kp.blockDim;
      st.smem = kp.sharedMemBytes;
      cudaLaunchAttributeValue v = {};
      if (cudaGraphKernelNodeGetAttribute(node, cudaKernelNodeAttributeClusterDimension, &v) == cudaSuccess &&
          v.clusterDim.x > 0)
        st.cluster = dim3(v.clusterDim.x, v.clusterDim.y, v.clusterDim.z);
      cudaGetLastError();
      st.args.resize(st.pk->arg_bytes);
      st.pk->pack(kp.kernelParams, st.args.data());
      chain.push_back(std::move(st));
    } else if (t == cudaGraphNodeTypeMemset) {
      PhaseStep st;
      st.memset = true;
      if (cudaGraphMemsetNodeGetParams(node, &st.ms) != cudaSuccess) {
        why = "memset node";
        ok = false;
        break;
      }
      chain.push_back(std::move(st));
    } else if (t != cudaGraphNodeTypeEmpty) {
      why = "a node of the schedule is neither a kernel nor a memset";
      ok = false;
      break;
    }
    // the edges of a captured schedule carry data (programmatic edges between the kernels), so
    // they are read with it
    size_t nd = 0;
    if (cudaGraphNodeGetDependentNodes(node, nullptr, nullptr, &nd) != cudaSuccess || nd > 1) {
      why = "the schedule is not a single chain";
      ok = false;
      break;
    }
    cudaGraphNode_t next = nullptr;
    cudaGraphEdgeData edge = {};
    if (nd == 1 && cudaGraphNodeGetDependentNodes(node, &next, &edge, &nd) != cudaSuccess) {
      why = "dependent node";
      ok = false;
      break;
    }
    node = nd == 1 ? next : nullptr;
  }
  cudaGraphDestroy(g);
  return ok;
}

// Builds b's graph in the phase layout.  Instances are taken longest schedule first; each joins
// the first group whose leader's chain agrees with its own step for step (a shorter schedule is
// a prefix of a longer one), else it leads a new group; each group is then dealt into `split`.  Step p of a group is one launch over
// its first n_p members (those with more than p steps) -- or their memsets -- after step p - 1;
// the groups are independent branches between a fork and a join.
bool build_phase_graph(fmg_batch* b, const std::vector<int>& csz, int split, std::string& why) {
  const int n = (int)b->cs.size();
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    why = "capture stream";
    return false;
  }
  std::vector<std::vector<PhaseStep>> chains(n);
  bool ok = true;
  for (int i = 0; i < n && ok; ++i) ok = phase_chain(b->cs[i], csz[i], cap, chains[i], why);
  cudaStreamDestroy(cap);
  if (!ok) return false;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return chains[x].size() > chains[y].size(); });
  std::vector<std::vector<int>> groups;
  for (int i : order) {
    bool placed = false;
    for (auto& gr : groups) {
      const auto& lead = chains[gr[0]];
      bool match = chains[i].size() <= lead.size();
      for (size_t p = 0; match && p < chains[i].size(); ++p) match = same_step(chains[i][p], lead[p]);
      if (match) {
        gr.push_back(i);
        placed = true;
        break;
      }
    }
    if (!placed) groups.push_back({i});
  }
  // each group dealt round-robin into `split` groups of similar level counts, which run as
  // parallel branches (the latency-bound phases of one overlap the streaming ones of another)
  if (split > 1) {
    std::vector<std::vector<int>> dealt;
    for (const auto& gr : groups) {
      const int parts = std::min(split, (int)gr.size());
      std::vector<std::vector<int>> sub(parts);
      for (size_t k = 0; k < gr.size(); ++k) sub[k % parts].push_back(gr[k]);
      for (auto& sg : sub) dealt.push_back(std::move(sg));
    }
    groups.swap(dealt);
  }
  // the active members of a group at step p (those with more than p steps: a prefix)
  auto active = [&](const std::vector<int>& gr, size_t p) {
    int k = 0;
    while (k < (int)gr.size() && chains[gr[k]].size() > p) ++k;
    return k;
  };
  cudaError_t e;
  cudaGraph_t g = nullptr;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) {
    why = std::string("graph: ") + cudaGetErrorString(e);
    return false;
  }
  auto bail = [&](cudaError_t err, const char* what) {
    why = std::string(what) + ": " + cudaGetErrorString(err);
    cudaGraphDestroy(g);
    return false;
  };
  cudaGraphNode_t fork = nullptr;
  if ((e = cudaGraphAddEmptyNode(&fork, g, nullptr, 0)) != cudaSuccess) return bail(e, "fork node");
  std::vector<cudaGraphNode_t> tails;
  int kernels = 0;
  for (size_t q = 0; q < groups.size(); ++q) {
    const auto& lead = chains[groups[q][0]];
    cudaGraphNode_t prev = fork;
    for (size_t p = 0; p < lead.size(); ++p) {
      const int na = active(groups[q], p);
      if (lead[p].memset) {
        std::vector<cudaGraphNode_t> ms(na);
        for (int k = 0; k < na; ++k)
          if ((e = cudaGraphAddMemsetNode(&ms[k], g, &prev, 1, &chains[groups[q][k]][p].ms)) != cudaSuccess)
            return bail(e, "memset node");
        cudaGraphNode_t join = nullptr;
        if ((e = cudaGraphAddEmptyNode(&join, g, ms.data(), ms.size())) != cudaSuccess) return bail(e, "join node");
        prev = join;
        continue;
      }
      const PhaseStep& st = lead[p];
      if (st.smem > 48 * 1024 &&
          (e = cudaFuncSetAttribute(st.pk->batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st.smem)) !=
              cudaSuccess)
        return bail(e, "phase kernel shared memory");
      if (st.cluster.x * st.cluster.y * st.cluster.z > 8 &&
          (e = cudaFuncSetAttribute(st.pk->batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
        return bail(e, "phase kernel cluster size");
      // one launch per `cap` members: its table (the kernel's parameter) holds their entries
      std::vector<cudaGraphNode_t> part;
      std::vector<unsigned char> tab((size_t)st.pk->cap * st.pk->arg_bytes);
      for (int k0 = 0; k0 < na; k0 += st.pk->cap) {
        const int nk = std::min(st.pk->cap, na - k0);
        std::fill(tab.begin(), tab.end(), (unsigned char)0);
        for (int k = 0; k < nk; ++k)
          std::memcpy(tab.data() + (size_t)k * st.pk->arg_bytes, chains[groups[q][k0 + k]][p].args.data(),
                      st.pk->arg_bytes);
        void* params[1] = {tab.data()};
        cudaKernelNodeParams kp = {};
        kp.func = const_cast<void*>(st.pk->batch);
        kp.gridDim = dim3(st.grid.x, st.grid.y, (unsigned)nk);
        kp.blockDim = st.block;
        kp.sharedMemBytes = st.smem;
        kp.kernelParams = params;
        cudaGraphNode_t nd = nullptr;
        if ((e = cudaGraphAddKernelNode(&nd, g, &prev, 1, &kp)) != cudaSuccess) return bail(e, "phase kernel node");
        if (st.cluster.x > 0) {
          cudaLaunchAttributeValue v = {};
          v.clusterDim.x = st.cluster.x;
          v.clusterDim.y = st.cluster.y;
          v.clusterDim.z = st.cluster.z;
          if ((e = cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributeClusterDimension, &v)) != cudaSuccess)
            return bail(e, "phase kernel cluster");
        }
        ++kernels;
        part.push_back(nd);
      }
      cudaGraphNode_t nd = part[0];
      if (part.size() > 1 && (e = cudaGraphAddEmptyNode(&nd, g, part.data(), part.size())) != cudaSuccess)
        return bail(e, "join node");
      prev = nd;
    }
    tails.push_back(prev);
  }
  cudaGraphNode_t join = nullptr;
  if ((e = cudaGraphAddEmptyNode(&join, g, tails.data(), tails.size())) != cudaSuccess) return bail(e, "join node");
  if ((e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess) {
    b->exec = nullptr;
    return bail(e, "phase graph instantiate");
  }
  b->graph = g;
  b->kernels = kernels;
  b->groups = (int)groups.size();
  b->mode = FMG_BATCH_PHASES;
  return true;
}

}  // namespace

void fmg::set_thread_error(const std::string& msg) { t_err = msg; }

// ============================================================================ C ABI

extern "C" {

void fmg_default_params(fmg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dim = 2;
  p->coarse_cells = 4;
  p->refinements = 4;
  p->f = FMG_F_CUBIC;
  p->f_scale = 1.0;
  p->m_vcycles = 2;
  p->nu_pre = 2;
  p->nu_post = 2;
  p->p_corrections = 1;
  p->precision = FMG_PREC_FP64;
  p->newton_tol = 1e-6;
  p->newton_maxit = 20;
  p->level1_tol = 1e-6;
  p->level1_maxit = 50;
  p->smoother = FMG_SMOOTHER_RBGS;
  p->nonlinear = FMG_NONLINEAR_NEWTON;
}

fmg_status fmg_workspace_bytes(const fmg_params* p, size_t* bytes) {
  if (const char* why = validate(p)) return fail(nullptr, FMG_ERR_INVALID, why);
  if (!bytes) return fail(nullptr, FMG_ERR_INVALID, "bytes is NULL");
  *bytes = layout(nullptr, p, nullptr);
  return FMG_OK;
}

fmg_status fmg_create(const fmg_params* p, const double* g_fine, int g_on_device, void* stream, void* workspace,
                      size_t workspace_bytes, fmg_ctx** out) {
  if (!out) return fail(nullptr, FMG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (const char* why = validate(p)) return fail(nullptr, FMG_ERR_INVALID, why);
  if (!g_fine) return fail(nullptr, FMG_ERR_INVALID, "g is NULL");
  fmg_ctx* c = new (std::nothrow) fmg_ctx();
  if (!c) return fail(nullptr, FMG_ERR_OOM, "host allocation failed");
  c->p = *p;
  c->nlev = p->refinements + 1;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess && !c->stream) {
    // graph capture needs a stream other than the legacy default stream
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    c->own_stream = (e == cudaSuccess);
  }
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return fail(nullptr, FMG_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  const size_t need = layout(c, p, nullptr);
  if (workspace) {
    if (workspace_bytes < need) {
      delete c;
      return fail(nullptr, FMG_ERR_INVALID, "workspace smaller than fmg_workspace_bytes");
    }
    c->arena = workspace;
    c->own_arena = false;
  } else {
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
      delete c;
      return fail(nullptr, FMG_ERR_CUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
    }
    if (need > free_b) {
      delete c;
      return fail(nullptr, FMG_ERR_OOM, "not enough free device memory for the level hierarchy");
    }
    e = cudaMalloc(&c->arena, need);
    if (e != cudaSuccess) {
      delete c;
      return fail(nullptr, FMG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->own_arena = true;
  }
  c->arena_bytes = need;
  layout(c, p, (char*)c->arena);
  c->cheb = cheb_coefficients();
  fmg_status s = FMG_OK;
  e = cudaMemsetAsync(c->arena, 0, need, c->stream);
  if (e != cudaSuccess) s = fail(c, FMG_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  if (s == FMG_OK) s = load_rhs(c, g_fine, g_on_device);
  // the coefficient table: FP64 as given, its FP32 rounding and its float-float split
  std::vector<double> coef64, coefff;
  std::vector<float> coef32;
  if (s == FMG_OK && p->coefficient) {
    const long long n = ipow(p->coarse_cells, p->dim) * p->dim;
    coef64.assign(p->coefficient, p->coefficient + n);
    coef32.resize(n);
    coefff.resize(n);
    for (long long i = 0; i < n; ++i) {
      const float hi = (float)coef64[i];
      const float lo = (float)(coef64[i] - (double)hi);
      coef32[i] = hi;
      std::memcpy(reinterpret_cast<char*>(&coefff[i]), &hi, 4);
      std::memcpy(reinterpret_cast<char*>(&coefff[i]) + 4, &lo, 4);
    }
    e = cudaMemcpyAsync((void*)c->vc.a64, coef64.data(), n * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)c->vc.a32, coef32.data(), n * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)c->vc.aff, coefff.data(), n * 8, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) s = fail(c, FMG_ERR_CUDA, std::string("coefficient upload: ") + cudaGetErrorString(e));
  }
  c->p.coefficient = nullptr;   // the caller's array is not kept
  if (s == FMG_OK) {
    e = launch_coarse_inverse(p->dim, c->geo[0], c->Ainv, c->st, c->stream, vcp(c));
    const long long n1 = ipow(p->coarse_cells - 1, p->dim);
    if (e == cudaSuccess) e = launch_to_f32(c->Ainv, c->Ainv32, n1 * n1, c->stream);
    if (e == cudaSuccess) e = launch_aug_jtab(p->dim, p->coarse_cells, (int*)c->ab.jtab, c->stream);
    if (e != cudaSuccess) s = fail(c, FMG_ERR_CUDA, std::string("coarse inverse: ") + cudaGetErrorString(e));
  }
  if (s == FMG_OK) s = read_state(c, nullptr, false);
  if (s != FMG_OK) {
    t_err = c->err;
    fmg_destroy(c);
    return s;
  }
  *out = c;
  return FMG_OK;
}

fmg_status fmg_set_rhs(fmg_ctx* c, const double* g_fine, int g_on_device) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  return load_rhs(c, g_fine, g_on_device);
}

fmg_status fmg_solve(fmg_ctx* c, double* u_out, int out_on_device, fmg_stats* st) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  if (fmg_status s = ensure_graph(c)) return s;
  CK(c, cudaGraphLaunch(c->gexec, c->stream));
  const int top = c->nlev - 1;
  if (u_out)
    CK(c, cudaMemcpyAsync(u_out, c->u[top], c->geo[top].nodes * sizeof(double),
                          out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (st || (u_out && !out_on_device)) return read_state(c, st, true);
  return FMG_OK;
}

fmg_status fmg_sync(fmg_ctx* c, fmg_stats* st) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  return read_state(c, st, true);
}

fmg_status fmg_solve_batch(fmg_ctx** cs, int count, double** u_outs, fmg_stats* sts) {
  if (!cs || count < 1) return fail(nullptr, FMG_ERR_INVALID, "bad batch arguments");
  for (int i = 0; i < count; ++i)
    if (!cs[i]) return fail(nullptr, FMG_ERR_INVALID, "NULL context in batch");
  fmg_batch* b = nullptr;
  fmg_status s = fmg_batch_create(cs, count, cs[0]->stream, &b);
  if (s != FMG_OK) return s;
  std::vector<fmg_stats> tmp(sts ? 0 : count);
  s = fmg_batch_solve(b, sts ? sts : tmp.data());
  if (s == FMG_OK && u_outs) {
    for (int i = 0; i < count && s == FMG_OK; ++i) {
      if (!u_outs[i]) continue;
      const int top = cs[i]->nlev - 1;
      cudaError_t e = cudaMemcpyAsync(u_outs[i], cs[i]->u[top], cs[i]->geo[top].nodes * sizeof(double),
                                      cudaMemcpyDeviceToDevice, b->launch);
      if (e != cudaSuccess) s = fail(nullptr, FMG_ERR_CUDA, std::string("batch output: ") + cudaGetErrorString(e));
    }
    cudaStreamSynchronize(b->launch);
  }
  fmg_batch_destroy(b);
  return s;
}

fmg_status fmg_batch_destroy(fmg_batch* b) {
  if (!b) return FMG_OK;
  if (b->launch) cudaStreamSynchronize(b->launch);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  if (b->own_launch && b->launch) cudaStreamDestroy(b->launch);
  delete b;
  return FMG_OK;
}

fmg_status fmg_batch_create(fmg_ctx** cs, int count, void* stream, fmg_batch** out) {
  return fmg_batch_create_mode(cs, count, stream, FMG_BATCH_AUTO, 0, out);
}

fmg_status fmg_batch_info(const fmg_batch* b, int* mode, int* kernel_nodes, int* groups) {
  if (!b) return fail(nullptr, FMG_ERR_INVALID, "batch is NULL");
  if (mode) *mode = b->mode;
  if (kernel_nodes) *kernel_nodes = b->kernels;
  if (groups) *groups = b->groups;
  return FMG_OK;
}

fmg_status fmg_batch_create_mode(fmg_ctx** cs, int count, void* stream, int mode, int phase_split,
                                 fmg_batch** out) {
  if (!out || !cs || count < 1) return fail(nullptr, FMG_ERR_INVALID, "bad batch arguments");
  if (mode != FMG_BATCH_AUTO && mode != FMG_BATCH_PHASES && mode != FMG_BATCH_BRANCHES)
    return fail(nullptr, FMG_ERR_INVALID, "unknown batch mode");
  if (phase_split < 0 || phase_split > 1024) return fail(nullptr, FMG_ERR_INVALID, "phase_split out of range");
  if (phase_split == 0) phase_split = kDefaultPhaseSplit;
  *out = nullptr;
  int dev = -1;
  for (int i = 0; i < count; ++i) {
    if (!cs[i]) return fail(nullptr, FMG_ERR_INVALID, "NULL context in batch");
    if (dev < 0) dev = cs[i]->device;
    if (cs[i]->device != dev) return fail(nullptr, FMG_ERR_INVALID, "batch contexts on different devices");
    if (cs[i]->vc.a64) return fail(nullptr, FMG_ERR_INVALID, "batches take A = I only (no coefficient)");
  }
  fmg_batch* b = new (std::nothrow) fmg_batch();
  if (!b) return fail(nullptr, FMG_ERR_OOM, "host allocation failed");
  b->cs.assign(cs, cs + count);
  auto bail = [&](cudaError_t e, const std::string& what) {
    fmg_batch_destroy(b);
    return fail(nullptr, FMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e;
  b->launch = (cudaStream_t)stream;
  if (!b->launch) {
    if ((e = cudaStreamCreateWithFlags(&b->launch, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "stream");
    b->own_launch = true;
  }
  b->events.resize(count + 1, nullptr);
  for (int i = 0; i <= count; ++i)
    if ((e = cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
  // cluster size of each instance's Newton kernel (outside the capture)
  std::vector<int> csz(count);
  for (int i = 0; i < count; ++i) {
    fmg_ctx* c = cs[i];
    csz[i] = aug_cluster_size(c->p.dim, c->p.coarse_cells, c->p.precision == FMG_PREC_MIXED, c->ab.smem);
    if (csz[i] < 1) {
      fmg_batch_destroy(b);
      return fail(nullptr, FMG_ERR_CUDA, "no usable thread-block cluster size for the batched Newton kernel");
    }
  }
  if (mode != FMG_BATCH_BRANCHES) {
    std::string why;
    if (build_phase_graph(b, csz, phase_split, why)) {
      *out = b;
      return FMG_OK;
    }
    if (mode == FMG_BATCH_PHASES) {
      fmg_batch_destroy(b);
      return fail(nullptr, FMG_ERR_INVALID, "no phase layout for this batch: " + why);
    }
    // fall back to branches
    cudaGetLastError();
  }
  b->mode = FMG_BATCH_BRANCHES;
  b->streams.resize(count, nullptr);
  for (int i = 0; i < count; ++i)
    if ((e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "stream");
  // one graph: fork on the launch stream, every instance's whole schedule on its own stream, join
  if ((e = cudaStreamBeginCapture(b->launch, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return bail(e, "begin capture");
  t_site = nullptr;
  int fail_at = -1;
  cudaError_t ce = cudaEventRecord(b->events[count], b->launch);
  for (int i = 0; i < count && ce == cudaSuccess; ++i) {
    fail_at = i;
    fmg_ctx* c = cs[i];
    ce = cudaStreamWaitEvent(b->streams[i], b->events[count], 0);
    if (ce != cudaSuccess) break;
    cudaStream_t saved = c->stream;
    const bool timing = c->timing;
    const int cluster = c->cluster_aug;
    c->stream = b->streams[i];
    c->cluster_aug = csz[i];
    c->timing = false;   // the batch graph carries no per-kernel timing events
    ce = run_fmg(c);
    c->timing = timing;
    c->cluster_aug = cluster;
    c->stream = saved;
    if (ce == cudaSuccess) ce = cudaEventRecord(b->events[i], b->streams[i]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->launch, b->events[i], 0);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->launch, &g);
  if (ce != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bail(ce != cudaSuccess ? ce : e,
                "batch capture (instance " + std::to_string(fail_at) + ")" +
                    (t_site ? std::string(" at ") + t_site : std::string()));
  }
  b->graph = g;
  if ((e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess) return bail(e, "batch instantiate");
  b->kernels = graph_kernel_nodes(g);
  *out = b;
  return FMG_OK;
}

fmg_status fmg_batch_solve(fmg_batch* b, fmg_stats* sts) {
  if (!b) return fail(nullptr, FMG_ERR_INVALID, "batch is NULL");
  // the instances' work waits for anything queued on their own streams before
  for (fmg_ctx* c : b->cs) {
    if (c->stream == b->launch) continue;
    cudaEvent_t ev = b->events[0];
    cudaError_t e = cudaEventRecord(ev, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->launch, ev, 0);
    if (e != cudaSuccess) return fail(nullptr, FMG_ERR_CUDA, std::string("batch ordering: ") + cudaGetErrorString(e));
  }
  cudaError_t e = cudaGraphLaunch(b->exec, b->launch);
  if (e != cudaSuccess) return fail(nullptr, FMG_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  // later work on the contexts' own streams sees the batch's results
  const int n = (int)b->cs.size();
  if ((e = cudaEventRecord(b->events[n], b->launch)) != cudaSuccess)
    return fail(nullptr, FMG_ERR_CUDA, std::string("batch ordering: ") + cudaGetErrorString(e));
  for (fmg_ctx* c : b->cs)
    if (c->stream != b->launch && (e = cudaStreamWaitEvent(c->stream, b->events[n], 0)) != cudaSuccess)
      return fail(nullptr, FMG_ERR_CUDA, std::string("batch ordering: ") + cudaGetErrorString(e));
  if (!sts) return FMG_OK;
  e = cudaStreamSynchronize(b->launch);
  if (e != cudaSuccess) return fail(nullptr, FMG_ERR_CUDA, std::string("batch sync: ") + cudaGetErrorString(e));
  fmg_status worst = FMG_OK;
  for (size_t i = 0; i < b->cs.size(); ++i) {
    fmg_status s = read_state(b->cs[i], &sts[i], true);
    if (s != FMG_OK && worst == FMG_OK) {
      worst = s;
      t_err = b->cs[i]->err;
    }
  }
  return worst;
}

fmg_status fmg_batch_sync(fmg_batch* b) {
  if (!b) return fail(nullptr, FMG_ERR_INVALID, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->launch);
  if (e != cudaSuccess) return fail(nullptr, FMG_ERR_CUDA, std::string("batch sync: ") + cudaGetErrorString(e));
  return FMG_OK;
}

fmg_status fmg_set_kernel_timing(fmg_ctx* c, int on) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  if ((on != 0) != c->timing) {
    CK(c, cudaStreamSynchronize(c->stream));
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->timing = on != 0;
  }
  return FMG_OK;
}

fmg_status fmg_debug_barrier_fault(fmg_ctx* c, long long spins, int skip_block) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  if (spins < 0 || skip_block < -1) return fail(c, FMG_ERR_INVALID, "bad arguments");
  CK(c, cudaStreamSynchronize(c->stream));
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  c->ab.bar_spins = spins;
  c->ab.bar_skip = skip_block;
  return FMG_OK;
}

fmg_status fmg_kernel_time(fmg_ctx* c, int kind, int level, double* total_ms, int* launches) {
  if (!c || !total_ms) return fail(c, FMG_ERR_INVALID, "bad arguments");
  CK(c, cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  int n = 0;
  for (size_t i = 0; i < c->timed_next && i < c->timed.size(); ++i) {
    const fmg_ctx::Timed& t = c->timed[i];
    if (t.kind != kind || (level != 0 && t.level != level)) continue;
    float ms = 0.0f;
    CK(c, cudaEventElapsedTime(&ms, t.e0, t.e1));
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  if (launches) *launches = n;
  return FMG_OK;
}

int fmg_graph_kernels(const fmg_ctx* c) { return c ? c->graph_kernels : -1; }

fmg_status fmg_autotune_augmented(fmg_ctx* c, int* tuned) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  if (tuned) *tuned = 0;
  if (c->cluster_aug > 0) return FMG_OK;   // the cluster variant's shape is fixed
  const bool mixed = c->p.precision == FMG_PREC_MIXED;
  // one solve: every level holds the iterate its augmented step meets
  fmg_status st = ensure_graph(c);
  if (st != FMG_OK) return st;
  CK(c, cudaMemsetAsync(c->st, 0, offsetof(DevState, alpha_cur), c->stream));
  CK(c, cudaGraphLaunch(c->gexec, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  double* pristine = nullptr;
  CK(c, cudaMalloc(&pristine, c->geo[c->nlev - 1].nodes * sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  int count = 0;
  const int last = c->nlev;
  for (int k = 2; k <= last && ce == cudaSuccess; ++k) {
    const LevelGeo g = c->geo[k - 1];
    // the level's iterate as the kernel finds it (mixed: float-float; the finest level's FP64
    // result is converted back)
    if (mixed && k == last)
      ce = launch_ff_from_f64(c->u[k - 1], pristine, g.nodes, c->stream);
    else
      ce = cudaMemcpyAsync(pristine, c->u[k - 1], g.nodes * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    const AugShape rule = aug_shape(c->p.dim, c->p.coarse_cells, k, mixed, c->ab, false);
    AugShape best = rule;
    float best_ms = 0.f;
    const int sfine = 1 << (k - 1);
    for (int chunk = 32; chunk >= 2 && ce == cudaSuccess; chunk >>= 1) {
      if (chunk > sfine) continue;
      for (int bpc = 1; bpc <= c->ab.bpc && ce == cudaSuccess; ++bpc) {
        set_aug_shape(c->p.dim, c->p.coarse_cells, k, mixed, AugShape{chunk, bpc});
        float ms_min = 0.f;
        for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep) {
          ce = cudaMemcpyAsync(c->u[k - 1], pristine, g.nodes * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
          if (ce == cudaSuccess) ce = cudaMemsetAsync(c->st, 0, offsetof(DevState, alpha_cur), c->stream);
          if (ce == cudaSuccess) ce = cudaEventRecord(e0, c->stream);
          if (ce == cudaSuccess)
            ce = launch_augmented(c->p.dim, c->p.coarse_cells, k, g, c->u[k - 1], mixed ? c->gf[k - 1] : c->g[k - 1],
                                  c->p.f, c->p.f_scale, c->p.newton_tol, c->p.newton_maxit, mixed, c->ab, c->st, k - 1,
                                  c->stream, 0, c->p.nonlinear == FMG_NONLINEAR_FIXED_POINT ? 1 : 0,
                                  mixed && k == last ? 1 : 0, vcp(c));
          if (ce == cudaSuccess) ce = cudaEventRecord(e1, c->stream);
          if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
          if (ce == cudaSuccess && (rep == 0 || ms < ms_min)) ms_min = ms;
        }
        if (ce == cudaSuccess && (best_ms == 0.f || ms_min < best_ms)) {
          best_ms = ms_min;
          best = AugShape{chunk, bpc};
        }
      }
    }
    if (ce == cudaSuccess) {
      set_aug_shape(c->p.dim, c->p.coarse_cells, k, mixed, best);
      ++count;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(pristine);
  // the trials leave the statistics and the level data of no solve: the next solve rebuilds both
  if (ce == cudaSuccess) ce = cudaMemsetAsync(c->st, 0, offsetof(DevState, alpha_cur), c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) return fail(c, FMG_ERR_CUDA, std::string("augmented autotune: ") + cudaGetErrorString(ce));
  // the next solve captures its graph again with the tuned shapes
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  if (tuned) *tuned = count;
  return FMG_OK;
}

fmg_status fmg_aug_shape(const fmg_ctx* c, int level, int* chunk, int* blocks_per_cell) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  if (level < 2 || level > c->nlev) return fail(nullptr, FMG_ERR_INVALID, "level out of range");
  const AugShape sh = aug_shape(c->p.dim, c->p.coarse_cells, level, c->p.precision == FMG_PREC_MIXED, c->ab,
                                c->cluster_aug == 0);
  if (chunk) *chunk = sh.chunk;
  if (blocks_per_cell) *blocks_per_cell = c->cluster_aug > 0 ? 1 : sh.bpc;
  return FMG_OK;
}

fmg_status fmg_autotune(fmg_ctx* c, int* tuned) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  if (tuned) *tuned = 0;
  if (c->p.smoother != FMG_SMOOTHER_CHEBYSHEV) return FMG_OK;   // the other kernels' shapes are fixed
  CK(c, cudaStreamSynchronize(c->stream));
  const bool mixed = c->p.precision == FMG_PREC_MIXED;
  const int top_cta = mixed ? coarse_cycle_top<float>(c) : coarse_cycle_top<double>(c);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(c, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, FMG_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
  }
  static const int kBlocks[] = {64, 128, 256, 512};
  static const int kStrips[] = {1, 2, 4, 8};
  int count = 0;
  for (int j = top_cta + 1; j <= c->nlev && ce == cudaSuccess; ++j) {
    const LevelGeo g = c->geo[j - 1];
    float best = 0.f;
    ChebShape best_sh = cheb_shape(c->p.dim, g.n, mixed ? 4 : 8);
    for (int bi = 0; bi < 4 && ce == cudaSuccess; ++bi)
      for (int si = 0; si < 4 && ce == cudaSuccess; ++si) {
        const ChebShape sh{kBlocks[bi], kStrips[si]};
        // time the kernel on the context's scratch arrays (their contents are rebuilt by
        // every solve): two warm-up launches, then five timed ones
        auto launch = [&]() -> cudaError_t {
          if (mixed)
            return launch_cheb_shaped<float>(c->p.dim, g, c->u32[j - 1], c->u32b[j - 1], c->d32[j - 1],
                                             c->u32[j - 1], c->cheb.cd[1], c->cheb.cr[1], false, sh, c->stream);
          return launch_cheb_shaped<double>(c->p.dim, g, c->ua[j - 1], c->dd[j - 1], c->b[j - 1], c->ua[j - 1],
                                            c->cheb.cd[1], c->cheb.cr[1], false, sh, c->stream);
        };
        for (int w = 0; w < 2 && ce == cudaSuccess; ++w) ce = launch();
        if (ce == cudaSuccess) ce = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 5 && ce == cudaSuccess; ++r) ce = launch();
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, c->stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce == cudaSuccess && (best == 0.f || ms < best)) {
          best = ms;
          best_sh = sh;
        }
      }
    if (ce == cudaSuccess) {
      set_cheb_shape(c->p.dim, g.n, mixed ? 4 : 8, best_sh);
      ++count;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return fail(c, FMG_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
  // the next solve captures its graph again with the tuned shapes
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  if (tuned) *tuned = count;
  return FMG_OK;
}

fmg_status fmg_tuned_shape(const fmg_ctx* c, int level, int* block, int* strip) {
  if (!c || level < 1 || level > c->nlev || !block || !strip) return fail(nullptr, FMG_ERR_INVALID, "bad arguments");
  const ChebShape sh = cheb_shape(c->p.dim, c->geo[level - 1].n, c->p.precision == FMG_PREC_MIXED ? 4 : 8);
  *block = sh.block;
  *strip = sh.strip;
  return FMG_OK;
}

fmg_status fmg_destroy(fmg_ctx* c) {
  if (!c) return FMG_OK;
  cudaStreamSynchronize(c->stream);
  for (auto& t : c->timed) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->own_arena && c->arena) cudaFree(c->arena);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return FMG_OK;
}

const char* fmg_last_error(const fmg_ctx* c) { return c ? c->err.c_str() : t_err.c_str(); }

int fmg_levels(const fmg_ctx* c) { return c ? c->nlev : -1; }

int fmg_level_cells(const fmg_ctx* c, int level) {
  if (!c || level < 1 || level > c->nlev) return -1;
  return c->geo[level - 1].n;
}

const double* fmg_solution(const fmg_ctx* c) { return c ? c->u[c->nlev - 1] : nullptr; }

// ------------------------------------------------------------------ component operations

fmg_status fmg_op_smooth(fmg_ctx* c, int level, const double* b, double* u, int sweeps, int order) {
  if (fmg_status s = check_level(c, level, 1)) return s;
  if (!b || !u || sweeps < 0) return fail(c, FMG_ERR_INVALID, "bad smoother arguments");
  if (c->p.smoother == FMG_SMOOTHER_CHEBYSHEV) {
    if (sweeps > kMaxCheb) return fail(c, FMG_ERR_INVALID, "Chebyshev smoothing takes at most 16 steps");
    CK(c, cheb_steps<double>(c, level, u, c->ua[level - 1], c->dd[level - 1], b, sweeps, false));
    return read_state(c, nullptr, false);
  }
  const int first = order ? 1 : 0;
  for (int i = 0; i < sweeps; ++i) {
    CK(c, launch_rbgs<double>(c->p.dim, c->geo[level - 1], u, b, first, c->stream, vcp(c)));
    CK(c, launch_rbgs<double>(c->p.dim, c->geo[level - 1], u, b, 1 - first, c->stream, vcp(c)));
  }
  return read_state(c, nullptr, false);
}

fmg_status fmg_op_smooth_f32(fmg_ctx* c, int level, const float* b, float* u, int sweeps, int order) {
  if (fmg_status s = check_level(c, level, 1)) return s;
  if (!b || !u || sweeps < 0) return fail(c, FMG_ERR_INVALID, "bad smoother arguments");
  if (c->p.smoother == FMG_SMOOTHER_CHEBYSHEV) {
    if (sweeps > kMaxCheb) return fail(c, FMG_ERR_INVALID, "Chebyshev smoothing takes at most 16 steps");
    if (!c->d32[level - 1]) return fail(c, FMG_ERR_INVALID, "FP32 Chebyshev smoothing needs a mixed-precision context");
    CK(c, cheb_steps<float>(c, level, u, c->u32b[level - 1], c->d32[level - 1], b, sweeps, false));
    return read_state(c, nullptr, false);
  }
  const int first = order ? 1 : 0;
  for (int i = 0; i < sweeps; ++i) {
    CK(c, launch_rbgs<float>(c->p.dim, c->geo[level - 1], u, b, first, c->stream, vcp(c)));
    CK(c, launch_rbgs<float>(c->p.dim, c->geo[level - 1], u, b, 1 - first, c->stream, vcp(c)));
  }
  return read_state(c, nullptr, false);
}

fmg_status fmg_op_residual(fmg_ctx* c, int level, const double* b, const double* u, double* r) {
  if (fmg_status s = check_level(c, level, 1)) return s;
  if (!b || !u || !r) return fail(c, FMG_ERR_INVALID, "NULL array");
  CK(c, launch_residual(c->p.dim, c->geo[level - 1], u, b, r, c->stream, vcp(c)));
  return read_state(c, nullptr, false);
}

fmg_status fmg_op_vcycle(fmg_ctx* c, int level, const double* b, double* u, int cycles) {
  if (fmg_status s = check_level(c, level, 1)) return s;
  if (!b || !u || cycles < 0) return fail(c, FMG_ERR_INVALID, "bad cycle arguments");
  c->timed_next = 0;
  for (int i = 0; i < cycles; ++i) CK(c, top_cycle(c, level, u, b));
  return read_state(c, nullptr, false);
}

fmg_status fmg_op_correction_step(fmg_ctx* c, int level, double* u, fmg_stats* st) {
  if (fmg_status s = check_level(c, level, 2)) return s;
  if (!u) return fail(c, FMG_ERR_INVALID, "NULL array");
  CK(c, cudaMemsetAsync(c->st, 0, offsetof(DevState, alpha_cur), c->stream));
  c->timed_next = 0;
  if (c->p.precision == FMG_PREC_MIXED) {
    // the mixed path works on float-float level data: u in, the step, u out
    const long long nodes = c->geo[level - 1].nodes;
    CK(c, launch_ff_from_f64(u, c->u[level - 1], nodes, c->stream));
    CK(c, correction_step_ff(c, level, false));
    CK(c, launch_ff_to_f64(c->u[level - 1], u, nodes, c->stream));
  } else {
    CK(c, correction_step(c, level, u));
  }
  return read_state(c, st, false);
}

fmg_status fmg_op_level1_solve(fmg_ctx* c, double* u, fmg_stats* st) {
  if (!c) return fail(nullptr, FMG_ERR_INVALID, "context is NULL");
  if (!u) return fail(c, FMG_ERR_INVALID, "NULL array");
  CK(c, cudaMemsetAsync(c->st, 0, offsetof(DevState, alpha_cur), c->stream));
  CK(c, launch_level1_newton(c->p.dim, c->geo[0], c->g[0], u, c->p.f, c->p.f_scale, c->p.level1_tol,
                             c->p.level1_maxit, c->p.precision == FMG_PREC_MIXED, c->st, c->stream, false,
                             vcp(c)));
  return read_state(c, st, false);
}

fmg_status fmg_op_prolong(fmg_ctx* c, int level, const double* u_coarse, double* u_fine) {
  if (fmg_status s = check_level(c, level, 2)) return s;
  if (!u_coarse || !u_fine) return fail(c, FMG_ERR_INVALID, "NULL array");
  CK(c, (launch_prolong<double, double>(c->p.dim, c->geo[level - 2], u_coarse, c->geo[level - 1], u_fine, 0,
                                        c->stream)));
  return read_state(c, nullptr, false);
}

}  // extern "C"

// ============================================================================ server services

namespace fmg {

cudaStream_t ctx_stream(const fmg_ctx* c) { return c->stream; }

size_t ctx_bytes(const fmg_ctx* c) { return c->arena_bytes; }

size_t ctx_fine_nodes(const fmg_ctx* c) { return (size_t)c->geo[c->nlev - 1].nodes; }

fmg_status ctx_make_concurrent(fmg_ctx* c) {
  const int cs = aug_cluster_size(c->p.dim, c->p.coarse_cells, c->p.precision == FMG_PREC_MIXED, c->ab.smem);
  if (cs < 1) return fail(c, FMG_ERR_CUDA, "no usable thread-block cluster size for the Newton kernel");
  if (cs != c->cluster_aug) {
    CK(c, cudaStreamSynchronize(c->stream));
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->cluster_aug = cs;
  }
  return FMG_OK;
}

fmg_status ctx_enqueue(fmg_ctx* c, const double* g_host, double* u_host, DevState* state_host) {
  if (fmg_status s = load_rhs(c, g_host, 0)) return s;
  if (fmg_status s = ensure_graph(c)) return s;
  const int top = c->nlev - 1;
  CK(c, cudaGraphLaunch(c->gexec, c->stream));
  CK(c, cudaMemcpyAsync(u_host, c->u[top], c->geo[top].nodes * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(state_host, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  return FMG_OK;
}

fmg_status ctx_decode(fmg_ctx* c, const DevState& h, fmg_stats* st) { return decode_state(c, h, 0u, st); }

const char* ctx_error(const fmg_ctx* c) { return c->err.c_str(); }

}  // namespace fmg

/*
 * fmg.h -- C ABI of the GB300 (sm_103a) full multigrid solver for semilinear
 * elliptic problems
 *
 *     -Laplace(u) + a f(u) = g  in Omega = (0,1)^d,  u = 0 on the boundary,
 *
 * discretized by P1 finite elements on nested, uniformly refined meshes
 * (2D: right triangles split along the (0,0)-(1,1) diagonal; 3D: Kuhn
 * tetrahedra), following H. Xie and F. Xu, "A full multigrid method for
 * semilinear elliptic equation" (arXiv 1611.05677):
 *
 *   - the model problem and its discretization: Sec. 2, eq. (2.1)-(2.7);
 *   - the nested mesh sequence T_H = T_{h_1} .. T_{h_n}, h_k = h_{k-1}/2:
 *     Sec. 3, eq. (3.1)-(3.3);
 *   - one correction step (linearized boundary value problem solved by m
 *     multigrid cycles, then the semilinear problem on V_H + span{u~}):
 *     Algorithm 3.1, eq. (3.4)-(3.6);
 *   - the full multigrid schedule: Algorithm 3.2.
 *
 * Discretization conventions (fixed by this library where the paper leaves
 * them open): h_1 = H; the pairings (f(x,u),v) and (g,v) use the vertex
 * (mass-lumped) rule on the current mesh, so the weight of an interior node is
 * h^d; the multigrid cycle is V(nu_pre, nu_post) with red-black Gauss-Seidel
 * (red = even i+j[+l]; pre-smoothing red then black, post-smoothing black then
 * red), restriction P^T, prolongation P (the natural inclusion of P1 spaces)
 * and an exact solve on level 1; the augmented problem (3.6) is solved by
 * Newton's method from (c, alpha) = (0, 1).
 *
 * Array layout.  Every nodal array of a level with n cells per side holds
 * (n+1)^d doubles (or floats), boundary nodes included, x fastest:
 * node (i, j[, l]) is at offset i + (n+1) (j + (n+1) l).  Boundary entries of
 * arrays the library writes are zero.
 *
 * Errors.  No function aborts, throws or exits.  Each returns an fmg_status;
 * the message of the last failure is available from fmg_last_error (per
 * context, or per thread for failures without a context).  All device waits
 * inside the library are bounded; a wait that runs out returns
 * FMG_ERR_TIMEOUT.  A context is bound to one CUDA stream and is not thread
 * safe; distinct contexts may be used from distinct threads.
 */
#ifndef FMG_H
#define FMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmg_ctx fmg_ctx;

typedef enum {
  FMG_OK = 0,
  FMG_ERR_INVALID = 1,         /* bad argument (sizes, enum values, NULL pointer) */
  FMG_ERR_OOM = 2,             /* not enough device memory (checked before allocating) */
  FMG_ERR_NO_CONVERGENCE = 3,  /* a Newton iteration hit its cap or its matrix was not SPD */
  FMG_ERR_NONFINITE = 4,       /* NaN/Inf in the data or in an iterate */
  FMG_ERR_TIMEOUT = 5,         /* a bounded device wait ran out */
  FMG_ERR_CUDA = 6             /* a CUDA runtime call failed; see fmg_last_error */
} fmg_status;

/* Nonlinearities a*f(u); all are monotone for a > 0 (Assumption A, eq. 2.5). */
typedef enum {
  FMG_F_CUBIC = 0,         /* a u^3               (Sec. 4, Example 1) */
  FMG_F_EXPM1 = 1,         /* a (exp(u) - 1) */
  FMG_F_LINEAR = 2,        /* a u                 (closed-form test case) */
  FMG_F_SIGNED_POW32 = 3,  /* a sign(u)|u|^{3/2}  (Sec. 4, Example 3) */
  FMG_F_NEG_EXP_NEG = 4    /* -a exp(-u)          (Sec. 4, Example 2) */
} fmg_nonlin;

typedef enum {
  FMG_PREC_FP64 = 0,   /* every step in FP64 */
  FMG_PREC_MIXED = 1   /* multigrid cycles in FP32 inside a defect correction whose level
                          iterate, right-hand side, residual and update are float-float (an
                          unevaluated sum of two FP32 numbers, ~48 significant bits); the
                          augmented Newton residual and its quadrature sums are float-float per
                          node and FP64 across nodes; the Newton Jacobians' per-node products
                          and the small factorizations (level 1 and eq. 3.6) are FP32, with the
                          chord iteration on eq. 3.6, which changes the convergence rate, not
                          the solution; the result is written as FP64 */
} fmg_precision;

typedef enum {
  FMG_SMOOTHER_RBGS = 0,       /* red-black Gauss-Seidel sweeps (nu_pre / nu_post sweeps) */
  FMG_SMOOTHER_CHEBYSHEV = 1   /* Chebyshev-Jacobi: the three-term Chebyshev iteration on D^{-1}A
                                  over [1/2, 2] (2 bounds that spectrum on these meshes), nu_pre /
                                  nu_post steps of one colour-free stencil pass each (<= 16) */
} fmg_smoother;

typedef enum {
  FMG_NONLINEAR_NEWTON = 0,      /* Newton on (3.6) (the mixed path: chord steps after the first) */
  FMG_NONLINEAR_FIXED_POINT = 1  /* fixed-point iteration on (3.6): the Galerkin stiffness on
                                    V_H + span{u~} implicit, f at the previous iterate; converges
                                    for nonlinearities that are mild against that stiffness */
} fmg_nonlinear_solver;

typedef struct {
  int dim;             /* 2 or 3 */
  int coarse_cells;    /* 1/H: cells per side of T_H; even; 2D <= 8, 3D <= 4 (the augmented
                          system of size N_H + 1 <= 50 is solved densely on one SM) */
  int refinements;     /* n - 1 >= 0: levels 1..refinements+1 (Sec. 3, eq. 3.1) */
  int f;               /* fmg_nonlin */
  double f_scale;      /* a > 0 */
  int m_vcycles;       /* m >= 1: multigrid cycles per correction step (Algorithm 3.1) */
  int nu_pre;          /* >= 0 pre-smoothing sweeps */
  int nu_post;         /* >= 0 post-smoothing sweeps */
  int p_corrections;   /* p >= 1: correction steps per level (Algorithm 3.2) */
  int precision;       /* fmg_precision */
  double newton_tol;   /* augmented Newton stops when ||delta||_inf <= tol max(1, ||y||_inf) */
  int newton_maxit;    /* augmented Newton iteration cap (<= 64) */
  double level1_tol;   /* same rule for the exact solve on level 1 */
  int level1_maxit;    /* level-1 Newton iteration cap (<= 64) */
  int smoother;        /* fmg_smoother of the multigrid cycles */
  int nonlinear;       /* fmg_nonlinear_solver of the augmented problem (3.6) */
  const double* coefficient;
                       /* the diffusion coefficient A(x) of eq. (2.1): NULL for A = I, or a host
                          array of coarse_cells^dim rows of dim doubles, the diagonal entries
                          (a_11, .., a_dd) of A on each cell of T_H (cell (cx, cy[, cz]) at row
                          cx + nc cy [+ nc^2 cz], nc = coarse_cells; entry order x, y[, z]).  A is
                          diagonal, SPD (every entry finite and > 0, else FMG_ERR_INVALID) and
                          constant on each coarse cell, so every level's P1 stiffness keeps the
                          (2d+1)-point pattern with a weight per mesh edge and the Galerkin
                          identity A_H = P^T A_h P holds level to level.  fmg_create copies the
                          array (the pointer is not kept).  Taken with the red-black smoother
                          only (FMG_SMOOTHER_CHEBYSHEV: FMG_ERR_INVALID); batches and the server
                          take A = I only. */
} fmg_params;

typedef struct {
  int levels;               /* n */
  int level1_iters;         /* Newton iterations of the level-1 solve */
  int newton_iters[32];     /* augmented Newton iterations on level k at index k-1 (summed over p) */
  double alpha[32];         /* final alpha of the last correction step on level k at index k-1 */
  unsigned int flags;       /* bit 0: a Newton cap was hit; bit 1: non-finite value; bit 2: u~
                               was (numerically) inside V_H and was dropped; bit 3: a matrix
                               was not SPD; bit 4: a device wait timed out */
} fmg_stats;

/* Defaults: dim 2, 1/H = 4, 4 refinements, cubic, a = 1, m = 2, nu = 2/2, p = 1 (the
 * schedule of Sec. 4: m = 2, p = 1), FP64, Newton tol 1e-6 / cap 20, level-1 tol 1e-6 /
 * cap 50.  Newton converges quadratically near the solution, so the update that passes the
 * 1e-6 test leaves an error of order 1e-12; in the mixed path the FP32 Jacobian and linear
 * solves make the convergence linear with a rate near 1e-6, leaving about 1e-12 as well. */
void fmg_default_params(fmg_params* p);

/* Device bytes one context needs for these parameters (the workspace size fmg_create
 * expects when the caller provides the memory).  Returns FMG_ERR_INVALID for bad params. */
fmg_status fmg_workspace_bytes(const fmg_params* p, size_t* bytes);

/* Creates a context for one problem.
 *   g_fine       nodal values of g on the finest mesh ((n_fine+1)^d doubles, layout above;
 *                boundary entries are ignored).  Host or device memory (g_on_device).  The
 *                library copies it; the caller keeps ownership of its buffer.
 *   stream       cudaStream_t (as void*) all work of this context is ordered on; NULL = the
 *                legacy default stream.
 *   workspace    device memory of at least fmg_workspace_bytes bytes that the context uses
 *                for all its arrays, owned by the caller and kept alive until fmg_destroy; or
 *                NULL, in which case the library allocates (cudaMalloc) and frees it itself.
 * On success *out receives the context.  Returns FMG_ERR_OOM when the device does not have
 * the memory (checked with cudaMemGetInfo before allocating). */
fmg_status fmg_create(const fmg_params* p, const double* g_fine, int g_on_device, void* stream,
                      void* workspace, size_t workspace_bytes, fmg_ctx** out);

/* Replaces g (same layout and ownership rules as fmg_create).  Host input is copied
 * through a pageable or pinned buffer as given; the copy is ordered on the context stream. */
fmg_status fmg_set_rhs(fmg_ctx* c, const double* g_fine, int g_on_device);

/* Runs Algorithm 3.2 and writes u_{h_n} ((n_fine+1)^d doubles, boundary zero) to u_out,
 * device or host memory (out_on_device).  The whole schedule is one CUDA graph, captured on
 * the first call and replayed afterwards.  With out_on_device = 1 and st = NULL the call is
 * asynchronous on the context stream and convergence problems are reported by the next call
 * that synchronizes (fmg_solve with st != NULL or host output, or fmg_sync).  Otherwise it
 * waits for the stream and checks the device status flags. */
fmg_status fmg_solve(fmg_ctx* c, double* u_out, int out_on_device, fmg_stats* st);

/* Waits for the context stream and returns the status accumulated by earlier asynchronous
 * solves (and fills st when non-NULL). */
fmg_status fmg_sync(fmg_ctx* c, fmg_stats* st);

/* Solves several independent problems (contexts created on the same device) at once, each
 * with its own u_out (device pointers, or NULL entries / NULL array to leave the results in
 * the contexts); a one-shot fmg_batch (below) ordered on the first context's stream.  Waits
 * for the work; sts (count entries) receives each instance's statistics when non-NULL. */
fmg_status fmg_solve_batch(fmg_ctx** cs, int count, double** u_outs, fmg_stats* sts);

/* A reusable batch: one CUDA graph that solves every instance once (Algorithm 3.2 for each).
 * The instances' augmented-space Newton kernels run on thread-block clusters (hardware
 * barriers, no cooperative launch), which many instances can run concurrently.  Two layouts:
 *
 *   FMG_BATCH_PHASES: level-synchronous phases.  Instances whose schedules agree launch for
 *     launch (same dimension, 1/H, precision, smoother, cycle and Newton settings; any number
 *     of refinements and any g and f_scale) form a group.  Stage k of Algorithm 3.2 (the
 *     correction step on level k) is the same sequence of kernels with the same grids for
 *     every member that has a level k, so each kernel of the stage is ONE launch over the
 *     work list of (instance, tile) items of all members still active at that stage (members
 *     sorted by their level count, so the active ones are a prefix): the kernel's own tiles in
 *     x and y, the instance in z, each instance's arguments read from a device table built at
 *     creation.  A solve is then as many launches as the longest member's schedule, per
 *     group, instead of the sum over instances.  2D only (the 3D kernels tile z).
 *   FMG_BATCH_BRANCHES: every instance's whole schedule is an independent branch on a
 *     stream of its own, so their kernels overlap on the device.
 *   FMG_BATCH_AUTO: PHASES when every instance's schedule is made of phase-batchable kernels
 *     (the 2D forms), BRANCHES otherwise.
 *
 * Both layouts run the same kernels with the same arguments for each instance, so they give
 * the same bits.  The contexts must stay alive and must not be solved on their own while a
 * batch solve is running; their results are at fmg_solution(ctx).  stream: the launch stream
 * (NULL: one the batch creates).  fmg_batch_create uses FMG_BATCH_AUTO. */
typedef struct fmg_batch fmg_batch;
typedef enum { FMG_BATCH_AUTO = 0, FMG_BATCH_PHASES = 1, FMG_BATCH_BRANCHES = 2 } fmg_batch_mode;
fmg_status fmg_batch_create(fmg_ctx** cs, int count, void* stream, fmg_batch** out);
/* mode: an fmg_batch_mode; FMG_BATCH_PHASES fails with FMG_ERR_INVALID (and a message naming
 * the first kernel that is not phase-batchable) instead of falling back to branches.
 * phase_split (phase layout): each set of instances whose schedules agree is dealt round-robin
 * (after sorting by level count) into that many groups, which run as parallel branches of
 * phases, so that one group's latency-bound phases (the Newton kernels, the one-CTA coarse
 * cycles) overlap another's streaming ones; 0: the default; 1..1024. */
fmg_status fmg_batch_create_mode(fmg_ctx** cs, int count, void* stream, int mode, int phase_split,
                                 fmg_batch** out);
/* The layout a batch uses (FMG_BATCH_PHASES or FMG_BATCH_BRANCHES), the kernel nodes of its
 * graph (launches per batch solve) and its number of phase groups (0 for branches); each
 * output may be NULL. */
fmg_status fmg_batch_info(const fmg_batch* b, int* mode, int* kernel_nodes, int* groups);
/* Launches the batch graph (after work already queued on the contexts' own streams).  With
 * sts == NULL it returns at once; otherwise it waits and fills count fmg_stats. */
fmg_status fmg_batch_solve(fmg_batch* b, fmg_stats* sts);
fmg_status fmg_batch_sync(fmg_batch* b);
fmg_status fmg_batch_destroy(fmg_batch* b);

/* Autotuner of launch shapes.  For a context with FMG_SMOOTHER_CHEBYSHEV it times every
 * candidate shape (threads per block 64..512 x nodes per thread along the outer axis 1..8)
 * of the Chebyshev step kernel on each of the context's levels that run it, on the
 * context's own scratch arrays, and keeps the fastest per (device, dimension, level size,
 * precision) for the whole process: every context on the device uses them from its next
 * graph capture (this context's captured graph is dropped).  Waits for the context stream
 * and must not overlap other work of the context.  *tuned (optional) receives the number of
 * levels tuned (0 for red-black smoothing, whose kernels have fixed shapes). */
fmg_status fmg_autotune(fmg_ctx* c, int* tuned);
/* Launch shape the context's Chebyshev step kernel uses on `level` (tuned or default). */
fmg_status fmg_tuned_shape(const fmg_ctx* c, int level, int* block, int* strip);
/* Autotuner of the augmented-space Newton kernel's launch shape (Algorithm 3.1 step 2, eq. 3.6):
 * for each level 2..n it solves once for the levels' iterates, then times every pair of column-
 * chunk length (2..32 fine nodes, a power of two within the column) and blocks per coarse cell
 * (1 up to the co-resident maximum of the cooperative launch) on a copy of that level's data,
 * and keeps the fastest per (device, dimension, 1/H, level, precision) for the whole process.
 * Unlike fmg_autotune this changes the order of the kernel's block sums, so results change in
 * rounding (a solve stays deterministic for a given shape).  Waits for the context stream, must
 * not overlap other work of the context, and leaves no solve's result in it.  Contexts on the
 * cluster variant (request server) keep their fixed shape.  *tuned: levels tuned (optional). */
fmg_status fmg_autotune_augmented(fmg_ctx* c, int* tuned);
/* Launch shape of the context's augmented kernel on `level` (2..n): chunk length and blocks
 * per coarse cell (tuned or the default rule). */
fmg_status fmg_aug_shape(const fmg_ctx* c, int level, int* chunk, int* blocks_per_cell);

/* Frees the context (and the workspace when the library allocated it).  NULL-safe. */
fmg_status fmg_destroy(fmg_ctx* c);

/* Message of the last failure on c, or of the calling thread when c is NULL. */
const char* fmg_last_error(const fmg_ctx* c);

/* Device pointer of the fine-level solution u_{h_n} inside the context ((n_fine+1)^d doubles,
 * layout above), valid until the next fmg_solve or fmg_destroy; NULL for a NULL context.  A
 * solve called with u_out = NULL leaves its result only here. */
const double* fmg_solution(const fmg_ctx* c);

/* Number of levels n and cells per side of level k (1-based), or -1 for bad arguments. */
int fmg_levels(const fmg_ctx* c);
int fmg_level_cells(const fmg_ctx* c, int level);

/* ---------------------------------------------------------------------------------------
 * Component operations.  They run one step of the method on caller-owned DEVICE arrays in
 * the nodal layout of the given level, ordered on the context stream, and wait for it.
 * They use the context's scratch arrays, so they must not overlap a running fmg_solve.
 * ------------------------------------------------------------------------------------- */

/* `sweeps` red-black Gauss-Seidel sweeps on A_k u = b at level k (the smoother of the
 * multigrid steps of Algorithm 3.1 step 1).  order 0: red then black; 1: black then red.
 * On a context with FMG_SMOOTHER_CHEBYSHEV: `sweeps` Chebyshev-Jacobi steps (order
 * ignored); the FP32 form then needs an FMG_PREC_MIXED context (its FP32 scratch). */
fmg_status fmg_op_smooth(fmg_ctx* c, int level, const double* b, double* u, int sweeps, int order);
fmg_status fmg_op_smooth_f32(fmg_ctx* c, int level, const float* b, float* u, int sweeps, int order);

/* r = b - A_k u at level k (the residual of the linear system of eq. 3.4). */
fmg_status fmg_op_residual(fmg_ctx* c, int level, const double* b, const double* u, double* r);

/* `cycles` V-cycles on A_k u = b from the initial guess in u (eq. 3.5), with the context's
 * nu_pre/nu_post and precision (FMG_PREC_MIXED: FP64 residual -> FP32 cycle -> FP64 update). */
fmg_status fmg_op_vcycle(fmg_ctx* c, int level, const double* b, double* u, int cycles);

/* One correction step u <- SemilinearMG(V_H, u, V_{h_k}) of Algorithm 3.1 at level k >= 2,
 * with the context's g (restricted to level k), m and precision.  u is FP64 in and out; an
 * FMG_PREC_MIXED context converts it to its float-float level data, takes the step as a mixed
 * solve does (FP32 cycles, float-float residual and update, chord iteration on eq. 3.6) and
 * converts back.  Newton iterations and alpha go to st (index k-1) when st is non-NULL. */
fmg_status fmg_op_correction_step(fmg_ctx* c, int level, double* u, fmg_stats* st);

/* Exact semilinear solve on level 1 (Algorithm 3.2 step 1) into u (level-1 layout). */
fmg_status fmg_op_level1_solve(fmg_ctx* c, double* u, fmg_stats* st);

/* u_fine = P_k u_coarse: the natural inclusion V_{h_{k-1}} -> V_{h_k} (eq. 3.3), k >= 2. */
fmg_status fmg_op_prolong(fmg_ctx* c, int level, const double* u_coarse, double* u_fine);

/* ---------------------------------------------------------------------------------------
 * Diagnostics: kernel timing inside the captured solve graph, and its size.
 * ------------------------------------------------------------------------------------- */

typedef enum {
  FMG_KT_AUGMENTED = 0,   /* the augmented-space Newton kernel of a correction step (eq. 3.6) */
  FMG_KT_SMOOTH_TOP = 1,  /* one smoothing step on the cycle's top level: a red-black sweep (both colours) or a Chebyshev step */
  FMG_KT_CORRECTION = 2,  /* a whole correction step (Algorithm 3.1) */
  FMG_KT_PRE_TOP = 3,     /* mixed path, 2D: fused pre-smoothing + residual + restriction, top level */
  FMG_KT_POST_TOP = 4     /* mixed path, 2D: fused prolongation + post-smoothing + update of the iterate, top level */
} fmg_kernel_kind;

/* on != 0: the next fmg_solve recaptures its graph with a pair of CUDA events around every
 * instrumented launch (event-record nodes; they add a little time to the solve).  on = 0
 * recaptures without them. */
fmg_status fmg_set_kernel_timing(fmg_ctx* c, int on);

/* Sum of the durations (ms) of the instrumented launches of `kind` in the most recent solve,
 * on `level` (1-based) or on all levels (level = 0), and their number.  Waits for the
 * context stream. */
fmg_status fmg_kernel_time(fmg_ctx* c, int kind, int level, double* total_ms, int* launches);

/* Kernel nodes in the captured solve graph (0 before the first solve, -1 for NULL). */
int fmg_graph_kernels(const fmg_ctx* c);

/* Failure-detection test hook (the paper has no counterpart: it exercises this library's
 * bounded device waits).  The augmented-space Newton kernel of a solve is one cooperative
 * launch whose blocks meet at a grid barrier after every pass; a waiting block polls at most
 * `spins` times (0 restores the default, 2^25) and then sets the timeout flag (fmg_stats.flags
 * bit 4) and an abort word that makes every block leave, so the solve returns FMG_ERR_TIMEOUT
 * instead of waiting without bound.  skip_block >= 0 makes that block skip its arrival at the
 * first barrier of every such launch, so the others run out of polls; -1 turns it off.  Nothing
 * faults or hangs: every wait is bounded.  The next solve recaptures its graph; a later solve
 * with the hook off starts from cleared barrier words and flags. */
fmg_status fmg_debug_barrier_fault(fmg_ctx* c, long long spins, int skip_block);

/* The current device's FP64 fused multiply-add rate, the roofline of the FP64 path's ALU-bound
 * kernels (the paper has no counterpart: it is a measurement service of this library).  Runs
 * `reps` (1..1000) timed launches of independent FMA chains, eight 256-thread blocks per SM,
 * and writes the rate in FP64 FLOP/s (an FMA counts as two) to *flops.  It allocates a few
 * bytes of device memory and a stream of its own, and waits for them. */
fmg_status fmg_fp64_fma_rate(int reps, double* flops);

/* ---------------------------------------------------------------------------------------
 * V-cycles that allocate no device memory.
 *
 * The paper has no counterpart to this entry point; it is a service of this library.  It is
 * for callers that cannot call cudaMalloc: code embedded in a host application whose own
 * memory pool owns the device memory and forbids raw allocations, latency-critical loops
 * where cudaMalloc/cudaFree would synchronize the device and stall other streams, and
 * programs that must know at load time that no allocation can fail later.  fmg_create needs
 * a workspace (its own or the caller's); this call needs none.
 *
 * It runs `cycles` FP64 V(nu_pre, nu_post) cycles on A_k u = b at level `level` (1-based; the
 * mesh of level k has coarse_cells * 2^(k-1) cells per side), always with red-black
 * Gauss-Seidel smoothing (nu_pre / nu_post are numbers of red-black sweeps) -- the same cycle
 * as fmg_op_vcycle on an FMG_PREC_FP64 context with FMG_SMOOTHER_RBGS (a Chebyshev context's
 * fmg_op_vcycle smooths differently).  b and u are the caller's DEVICE arrays in the
 * level-k nodal layout ((n+1)^d doubles, boundary entries zero); u holds the initial guess
 * and receives the result.  All coarser levels and the dense level-1 inverse live in one
 * file-scope device array of FMG_VCYCLE_NOALLOC_MAX_BYTES bytes, which every GPU that loads
 * the library holds until the process exits.  A size whose coarser levels do not fit (2D
 * levels up to 1024 cells per side fit, 3D up to 128) is rejected with FMG_ERR_INVALID; the
 * message is in fmg_last_error(NULL).
 *
 * The first call on a device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture on the device.  The
 * first call for a (dim, coarse_cells) pair also computes A_1^{-1} into the array.  Both are
 * kept per device index for the life of the process, so the call supports only the device's
 * primary context (the one the CUDA runtime and PyTorch use): after cudaDeviceReset, or from a
 * context created with the driver API, the kept address would not be valid.  Every
 * call shares the array, which keeps the last call's contents; the call clears the parts that
 * must start at zero itself.  Calls that overlap on the GPU (on different streams, or from
 * different threads on one device) race on the array and give wrong results.  The call only
 * queues work on `stream` (cudaStream_t, NULL = legacy default stream) and returns; u is
 * final when the stream reaches that point.
 */
#define FMG_VCYCLE_NOALLOC_MAX_BYTES ((size_t)8 << 20)
fmg_status fmg_vcycle_noalloc(int dim, int coarse_cells, int level, const double* b, double* u, int cycles,
                              int nu_pre, int nu_post, void* stream);

/* ---------------------------------------------------------------------------------------
 * Request server: continuous batching of independent solves on the current device.
 *
 * The paper solves one problem at a time; this is a serving layer over Algorithm 3.2.  A
 * worker thread admits queued requests in arrival order as soon as one of max_inflight
 * slots is free and the level hierarchy of the request fits the device memory budget
 * (idle cached contexts of other shapes are destroyed, least recently used first, to make
 * room).  Each admitted request runs on a context of its own shape: an idle cached one when
 * there is one (its hierarchy and captured graph stay on the device between requests), else
 * a new one.  Requests in flight overlap on the device; their augmented-space Newton kernels
 * run on thread-block clusters, which any number of solves may run side by side.  A request
 * gives the same bits whether it runs alone or among others.
 * ------------------------------------------------------------------------------------- */
typedef struct fmg_server fmg_server;

typedef struct {
  size_t hbm_budget;   /* device bytes the cached hierarchies may hold; 0 = 80% of the free
                          memory at creation */
  int max_inflight;    /* requests on the device at once, 1..64; 0 = 8 */
  int poll_us;         /* worker's pause between completion polls while requests are in
                          flight, microseconds; 0 = 20 */
} fmg_server_config;

typedef struct {
  unsigned long long ticket;  /* as returned by fmg_server_submit */
  fmg_status status;          /* FMG_ERR_OOM: the hierarchy alone exceeds the budget */
  fmg_stats stats;
  double queue_ms;            /* submit -> launch on the device (host clock) */
  double latency_ms;          /* submit -> result in u_host (host clock) */
} fmg_server_result;

typedef struct {
  size_t hbm_budget, bytes_held;
  int contexts_cached, in_flight, queued;
  size_t submitted, completed;
  int contexts_created, contexts_evicted;
} fmg_server_info;

/* Starts a server (and its worker thread) on the current device. */
fmg_status fmg_server_create(const fmg_server_config* cfg, fmg_server** out);
/* Queues one solve.  p as for fmg_create; g_host: nodal g on the finest mesh; u_host receives
 * u_{h_n}.  Both are HOST buffers ((n_fine+1)^d doubles) that must stay valid until the
 * request's result has been polled; pinned memory makes the copies asynchronous.  Returns at
 * once; *ticket identifies the request. */
fmg_status fmg_server_submit(fmg_server* s, const fmg_params* p, const double* g_host, double* u_host,
                             unsigned long long* ticket);
/* Moves up to max finished requests into out (completion order); returns how many. */
int fmg_server_poll(fmg_server* s, fmg_server_result* out, int max);
/* Waits until every submitted request has finished (results stay available to poll), at most
 * timeout_s seconds (FMG_ERR_TIMEOUT). */
fmg_status fmg_server_drain(fmg_server* s, double timeout_s);
fmg_status fmg_server_get_info(fmg_server* s, fmg_server_info* info);
/* Message of the calling thread's last server failure: a failed server call of this thread, or
 * the latest failed request that fmg_server_poll returned to it. */
const char* fmg_server_last_error(void);
/* Finishes the submitted requests, stops the worker and frees every cached hierarchy. */
fmg_status fmg_server_destroy(fmg_server* s);

#ifdef __cplusplus
}
#endif

#endif /* FMG_H */

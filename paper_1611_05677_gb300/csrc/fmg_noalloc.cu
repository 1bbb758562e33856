// V-cycles that allocate no device memory: every coarser level and the dense level-1 inverse
// live in one file-scope __device__ array of fixed size.  For callers that cannot call
// cudaMalloc (see fmg_vcycle_noalloc in include/fmg.h).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "fmg_internal.cuh"

namespace fmg {
namespace {

constexpr size_t kNoAllocBytes = FMG_VCYCLE_NOALLOC_MAX_BYTES;  // held by every GPU that loads the library

// The scratch itself.  Host code must not use this name as a device address (in host code it
// is only a stand-in); the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};   // device address of the scratch, per device
int g_ainv_key[kMaxDevices] = {};                  // (dim, coarse_cells) whose A_1^{-1} the scratch holds

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Layout inside the scratch: DevState | A_1^{-1} | u_1, b_1 | ... | u_{k-1}, b_{k-1}.
struct Layout {
  size_t state, ainv, levels, level_off[kMaxLevels], end;
};

Layout make_layout(int dim, int coarse_cells, int level) {
  Layout L{};
  size_t off = 0;
  L.state = off;
  off += align256(sizeof(DevState));
  const long long m = coarse_cells - 1;
  const long long N1 = ipow(m, dim);
  L.ainv = off;
  off += align256((size_t)(N1 * N1) * sizeof(double));
  L.levels = off;
  for (int j = 1; j < level; ++j) {
    L.level_off[j - 1] = off;
    const long long nodes = ipow((long long)(coarse_cells << (j - 1)) + 1, dim);
    off += align256(2 * (size_t)nodes * sizeof(double));
  }
  L.end = off;
  return L;
}

struct Ctx {
  int dim, nc, nu_pre, nu_post;
  cudaStream_t s;
  unsigned char* base;
  Layout lay;
  double* ainv;
  LevelGeo geo(int j) const {
    LevelGeo g;
    g.n = nc << (j - 1);
    g.np = g.n + 1;
    g.nodes = ipow(g.np, dim);
    return g;
  }
  double* u(int j) const { return reinterpret_cast<double*>(base + lay.level_off[j - 1]); }
  double* b(int j) const { return u(j) + geo(j).nodes; }
};

// Largest level the one-CTA coarse cycle takes (same rule as the context's schedule).
int coarse_top(const Ctx& c, int level) {
  const int nmax = c.dim == 2 ? 64 : 16;
  int j = 1;
  while (j < level && c.geo(j + 1).n <= nmax && coarse_cycle_smem<double>(c.dim, c.nc, j + 1, false) <= 200 * 1024) ++j;
  return j;
}

cudaError_t vcycle(const Ctx& c, int j, int level, double* u, const double* b) {
  cudaError_t e;
  if (j == 1) return launch_coarse_solve_f64(c.dim, c.geo(1), c.ainv, b, u, c.s);
  if (j <= coarse_top(c, level))
    return launch_coarse_cycle<double>(c.dim, c.nc, j, u, b, c.nu_pre, c.nu_post, c.ainv, nullptr, nullptr, false,
                                       c.s);
  const LevelGeo gf = c.geo(j), gc = c.geo(j - 1);
  for (int it = 0; it < c.nu_pre; ++it) {
    if ((e = launch_rbgs<double>(c.dim, gf, u, b, 0, c.s)) != cudaSuccess) return e;
    if ((e = launch_rbgs<double>(c.dim, gf, u, b, 1, c.s)) != cudaSuccess) return e;
  }
  if ((e = launch_residual_restrict<double, double>(c.dim, gf, u, b, gc, c.b(j - 1), c.u(j - 1), c.s)) !=
      cudaSuccess)
    return e;
  if ((e = vcycle(c, j - 1, level, c.u(j - 1), c.b(j - 1))) != cudaSuccess) return e;
  if ((e = launch_prolong<double, double>(c.dim, gc, c.u(j - 1), gf, u, 1, c.s)) != cudaSuccess) return e;
  for (int it = 0; it < c.nu_post; ++it) {
    if ((e = launch_rbgs<double>(c.dim, gf, u, b, 1, c.s)) != cudaSuccess) return e;
    if ((e = launch_rbgs<double>(c.dim, gf, u, b, 0, c.s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

fmg_status fail(fmg_status s, const std::string& m) {
  set_thread_error(m);
  return s;
}

}  // namespace
}  // namespace fmg

using namespace fmg;

extern "C" fmg_status fmg_vcycle_noalloc(int dim, int coarse_cells, int level, const double* b, double* u,
                                         int cycles, int nu_pre, int nu_post, void* stream) {
  if (dim != 2 && dim != 3) return fail(FMG_ERR_INVALID, "dim must be 2 or 3");
  if (coarse_cells < 2 || (coarse_cells & 1) || (dim == 2 && coarse_cells > 8) || (dim == 3 && coarse_cells > 4))
    return fail(FMG_ERR_INVALID, "coarse_cells must be even, 2D <= 8, 3D <= 4");
  if (level < 1 || level > kMaxLevels - 1) return fail(FMG_ERR_INVALID, "level out of range");
  if (!b || !u || cycles < 0 || nu_pre < 0 || nu_post < 0 || nu_pre > 64 || nu_post > 64)
    return fail(FMG_ERR_INVALID, "bad arguments");
  const Layout lay = make_layout(dim, coarse_cells, level);
  if (lay.end > kNoAllocBytes)
    return fail(FMG_ERR_INVALID, "level " + std::to_string(level) + " needs " + std::to_string(lay.end) +
                                     " bytes of scratch; the no-allocation V-cycle holds at most " +
                                     std::to_string(kNoAllocBytes) + " bytes");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(FMG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(FMG_ERR_INVALID, "device index out of range");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  bool need_inverse = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      // once per device, with that device current: the scratch's device address
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(FMG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_scratch_ptr[dev];
    const int key = dim * 100 + coarse_cells;
    if (g_ainv_key[dev] != key) {
      need_inverse = true;
      g_ainv_key[dev] = key;
    }
  }
  Ctx c;
  c.dim = dim;
  c.nc = coarse_cells;
  c.nu_pre = nu_pre;
  c.nu_post = nu_post;
  c.s = s;
  c.base = base;
  c.lay = lay;
  c.ainv = reinterpret_cast<double*>(base + lay.ainv);
  if (need_inverse) {
    e = cudaMemsetAsync(base + lay.state, 0, sizeof(DevState), s);
    if (e == cudaSuccess)
      e = launch_coarse_inverse(dim, c.geo(1), c.ainv, reinterpret_cast<DevState*>(base + lay.state), s);
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lk(g_mu);
      g_ainv_key[dev] = 0;
      return fail(FMG_ERR_CUDA, std::string("level-1 inverse: ") + cudaGetErrorString(e));
    }
  }
  // coarser levels' boundary rings must read as zero: clear the level region
  if (lay.end > lay.levels) {
    e = cudaMemsetAsync(base + lay.levels, 0, lay.end - lay.levels, s);
    if (e != cudaSuccess) return fail(FMG_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i < cycles; ++i) {
    e = vcycle(c, level, level, u, b);
    if (e != cudaSuccess) return fail(FMG_ERR_CUDA, std::string("V-cycle launch: ") + cudaGetErrorString(e));
  }
  return FMG_OK;
}

// Phase-batched launches.  A kernel that can run for many instances in one launch has its body
// as a __device__ function with the kernel's own parameter list; the kernel itself calls the
// body, and k_phase calls it once per instance with that instance's arguments, read from a
// table indexed by blockIdx.z (the grid's x and y are the kernel's own tiling, z is the
// instance) that is the launch's own parameter.  PhaseKernel records the pair and how to pack
// one launch's arguments (as a graph node holds them: one pointer per parameter) into a table
// entry.
#pragma once

#include <cuda_runtime.h>

#include <cuda/std/tuple>
#include <cstddef>
#include <new>
#include <utility>
#include <vector>

namespace fmg {

struct PhaseKernel {
  const void* solo;     // the kernel as launched for one instance
  const void* batch;    // k_phase over the same body
  size_t arg_bytes;     // bytes of one table entry
  size_t arg_align;     // its alignment
  int cap;              // entries of the table (k_phase's parameter: instances per launch at most)
  void (*pack)(void* const* params, void* dst);
};

// Bytes of kernel parameter space a phase table may take (the limit is 32764).
constexpr size_t kPhaseParamBytes = 32000;

template <typename T, int CAP>
struct PhaseTable {
  T e[CAP];
};

// The table is the kernel's own parameter (constant bank, read in place: __grid_constant__), so
// each block reads its instance's arguments as a solo launch reads its parameters.
template <auto Body, int MAXT, int MINB, typename... A>
__global__ void __launch_bounds__(MAXT, MINB)
    k_phase(const __grid_constant__ PhaseTable<cuda::std::tuple<A...>,
                                              (int)(kPhaseParamBytes / sizeof(cuda::std::tuple<A...>))> tab) {
  cuda::std::apply([](const auto&... a) { Body(a...); }, tab.e[blockIdx.z]);
}

template <typename... A, size_t... I>
void phase_pack(void* const* p, void* dst, std::index_sequence<I...>) {
  new (dst) cuda::std::tuple<A...>(*static_cast<A*>(p[I])...);
}

// The entry for kernel `solo` whose body is Body; MAXT, MINB: the launch bounds of the batched
// kernel (at least the block size the kernel is launched with).
template <auto Body, int MAXT, int MINB, typename... A>
PhaseKernel phase_kernel(void (*solo)(A...)) {
  PhaseKernel k;
  k.solo = (const void*)solo;
  k.batch = (const void*)&k_phase<Body, MAXT, MINB, A...>;
  k.arg_bytes = sizeof(cuda::std::tuple<A...>);
  k.arg_align = alignof(cuda::std::tuple<A...>);
  k.cap = (int)(kPhaseParamBytes / sizeof(cuda::std::tuple<A...>));
  k.pack = [](void* const* p, void* dst) { phase_pack<A...>(p, dst, std::index_sequence_for<A...>{}); };
  return k;
}

// The phase-batchable kernels of each translation unit (2D forms of the solve's kernels).
void phase_kernels_stencil(std::vector<PhaseKernel>& out);
void phase_kernels_ff(std::vector<PhaseKernel>& out);
void phase_kernels_fused(std::vector<PhaseKernel>& out);
void phase_kernels_newton(std::vector<PhaseKernel>& out);

}  // namespace fmg

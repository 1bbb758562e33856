// Diagnostics for the roofline of the FP64 path: the device's FP64 fused multiply-add rate.
//
// The FP64 path's augmented-space kernel and red-black sweeps issue several FP64 operations per
// byte they move, so their bound is the FP64 pipe, not HBM.  Its rate on this GPU is a small
// fraction of the FP32 rate and is not among the copy and GEMM peaks measured elsewhere, so it is
// measured here: every thread runs kChains independent FMA chains (x <- x a + b, a just below 1,
// which keeps the values bounded), enough warps per SM to cover the FMA latency, timed with CUDA
// events over several launches.
#include <cuda_runtime.h>

#include <string>

#include "fmg_internal.cuh"

namespace fmg {
namespace {

constexpr int kChains = 8;
constexpr int kSteps = 2048;

__global__ void __launch_bounds__(256) k_fp64_fma(double* out, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
  for (int s = 0; s < kSteps; ++s) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += x[c];
  // keeps the chains live; the value is never 1e300
  if (acc == 1e300) out[blockIdx.x] = acc;
}

}  // namespace
}  // namespace fmg

using namespace fmg;

extern "C" fmg_status fmg_fp64_fma_rate(int reps, double* flops) {
  if (!flops || reps < 1 || reps > 1000) {
    set_thread_error("fmg_fp64_fma_rate: reps must be in 1..1000 and flops non-NULL");
    return FMG_ERR_INVALID;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* out = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * 8 * (size_t)sms);
  const unsigned grid = 8u * (unsigned)sms;   // eight 256-thread blocks per SM
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_fp64_fma<<<grid, 256, 0, s>>>(out, 0.9999999, 1e-7);   // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; e == cudaSuccess && r < reps; ++r) {
    k_fp64_fma<<<grid, 256, 0, s>>>(out, 0.9999999, 1e-7);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    set_thread_error(std::string("fmg_fp64_fma_rate: ") + cudaGetErrorString(e));
    return FMG_ERR_CUDA;
  }
  const double fmas = (double)grid * 256.0 * kChains * kSteps * reps;
  *flops = 2.0 * fmas / (ms * 1e-3);
  return FMG_OK;
}

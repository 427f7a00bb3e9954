// kernels_peak.cu -- the FP32 SIMT fused multiply-add rate of this GPU, the
// denominator of the plain FP32 path's roofline (its synthesis and adjoint
// are FFMA-bound correlations).  Every thread runs 8 independent FMA chains
// (enough to cover the FMA pipe's latency), 512 threads per block, 4 blocks
// per SM; the result of every chain is written out so that none of the
// arithmetic can be dropped.
#include "../../include/scsc_diag.h"

#include <cuda_runtime.h>

namespace scsc {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 512;

__global__ void __launch_bounds__(kThreads) ffma_rate_kernel(float *sink, int iters, float a,
                                                             float b) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1e-3f * (float)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  sink[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace scsc

extern "C" scsc_status scsc_diag_ffma_peak(double *tflops, double *ms) {
  using namespace scsc;
  if (!tflops) return SCSC_EINVAL;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SCSC_ECUDA;
  const int blocks = 4 * n_sm;
  const int iters = 4096;
  float *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess)
    return SCSC_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  scsc_status st = SCSC_OK;
  float best = 0.0f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = SCSC_ECUDA;
  } else {
    // one warm-up launch, then the fastest of five timed ones
    ffma_rate_kernel<<<blocks, kThreads>>>(sink, iters, 0.999f, 1e-4f);
    for (int r = 0; r < 5 && st == SCSC_OK; ++r) {
      float t = 0.0f;
      if (cudaEventRecord(e0) != cudaSuccess) st = SCSC_ECUDA;
      ffma_rate_kernel<<<blocks, kThreads>>>(sink, iters, 0.999f, 1e-4f);
      if (st == SCSC_OK && (cudaEventRecord(e1) != cudaSuccess ||
                            cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        st = SCSC_ECUDA;
      if (st == SCSC_OK && (best == 0.0f || t < best)) best = t;
    }
    if (st == SCSC_OK && cudaGetLastError() != cudaSuccess) st = SCSC_ECUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (st != SCSC_OK || best <= 0.0f) return st == SCSC_OK ? SCSC_ECUDA : st;
  const double flops = 2.0 * (double)blocks * kThreads * (double)iters * kUnroll * kChains;
  *tflops = flops / ((double)best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return SCSC_OK;
}

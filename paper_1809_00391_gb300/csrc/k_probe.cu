// Device capability probes used by the benchmark: the FP64 fused
// multiply-add throughput of this GPU (the bound of the FP64 tracker, whose
// push is limited by the FP64 pipe rather than by memory).
#include <cuda_runtime.h>

#include "../../include/mbt.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;   // independent accumulators per thread: enough to cover the DFMA latency

// Every thread runs kChains independent chains of `iters` DFMAs each on
// values that stay finite (x <- x * a + b with |a| < 1); the result is stored
// so that nothing is eliminated.
__global__ void __launch_bounds__(kProbeThreads) k_dfma(int iters, double a, double b, double *sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // every chain stays in (0, 300) for these inputs, so this store never
  // happens; the compiler cannot know that, so the chains are kept
  if (sink != nullptr && s < 0.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" mbt_status mbt_probe_fp64_fma(int blocks_per_sm, int iters, int repeats, void *stream, double *flops_per_s,
                                         int *sms) {
  if (blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1 || iters > (1 << 24) || repeats < 1 || !flops_per_s)
    return MBT_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MBT_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = nsm * blocks_per_sm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MBT_ERR_CUDA;
  k_dfma<<<grid, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-6, nullptr);   // warm-up
  cudaEventRecord(e0, s);
  for (int r = 0; r < repeats; ++r) k_dfma<<<grid, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-6, nullptr);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return MBT_ERR_CUDA;
  *flops_per_s = 2.0 * (double)grid * kProbeThreads * kChains * (double)iters * repeats / (ms * 1e-3);
  if (sms) *sms = nsm;
  return MBT_OK;
}

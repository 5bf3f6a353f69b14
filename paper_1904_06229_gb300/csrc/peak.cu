// FP64 fused-multiply-add throughput probe: the denominator of the walk
// kernels' "fraction of FP64 peak".  Eight independent DFMA chains per thread
// over every SM; the result is written so nothing is optimised away.
#include <cuda_runtime.h>

#include "perm.h"
#include "perm_internal.h"

namespace perm {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_dfma_probe(double* sink, int iters, double a, double b) {
  double x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

void preload_peak_kernels() { load_kernel(k_dfma_probe); }

cudaError_t dfma_probe_launch(double* sink, int blocks, int iters, cudaStream_t stream) {
  k_dfma_probe<<<blocks, kProbeThreads, 0, stream>>>(sink, iters, 0.999999, 1e-7);
  return cudaGetLastError();
}

}  // namespace perm

extern "C" int perm_fp64_peak(double* gops) {
  using namespace perm;
  if (!gops) return PERM_ENULL;
  int count = 0, dev = 0, sms = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) return PERM_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERM_ECUDA;
  const int blocks = sms * 8;
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * blocks * kProbeThreads) != cudaSuccess) return PERM_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = PERM_OK;
  float best = 1e30f;
  const int iters = 4000;
  if (dfma_probe_launch(sink, blocks, iters / 8, nullptr) != cudaSuccess) rc = PERM_ECUDA;
  for (int rep = 0; rep < 5 && rc == PERM_OK; ++rep) {
    cudaEventRecord(e0, nullptr);
    if (dfma_probe_launch(sink, blocks, iters, nullptr) != cudaSuccess) rc = PERM_ECUDA;
    cudaEventRecord(e1, nullptr);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = PERM_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0.f && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (rc != PERM_OK) return rc;
  const double ops = (double)blocks * kProbeThreads * kProbeChains * (double)iters;
  *gops = ops / (best * 1e-3) / 1e9;
  return PERM_OK;
}

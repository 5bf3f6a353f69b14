// Pipe throughput probes: the denominators of the walk kernels' roofline
// fractions.  Each probe runs eight independent dependency chains of one
// instruction kind per thread over every SM (8 blocks of 256 threads per SM)
// and reports lane instructions per second; the result is written so nothing
// is optimised away.  The integer probes go through inline PTX so that the
// compiler cannot fold the chains algebraically.
//
//   PERM_PIPE_DFMA   FP64 fused multiply-add (register operands)
//   PERM_PIPE_FFMA   FP32 fused multiply-add
//   PERM_PIPE_FFMA2  packed FP32 fused multiply-add (two FMAs per lane)
//   PERM_PIPE_IMAD   32-bit integer multiply-add
//   PERM_PIPE_ALU    32-bit three-input logic op (LOP3)
//   PERM_PIPE_ISSUE  one packed FP32 FMA and one logic op per step, chains of
//                    both kinds interleaved: the rate at which the schedulers
//                    issue a stream that no single pipe bounds
#include <cuda_runtime.h>

#include "perm.h"
#include "perm_internal.h"

namespace perm {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

template <int PIPE>
__global__ void __launch_bounds__(kProbeThreads) k_pipe_probe(double* sink, int iters, double a, double b) {
  const int t = threadIdx.x;
  double s = 0.0;
  if constexpr (PIPE == PERM_PIPE_DFMA) {
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = t * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
    }
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
  } else if constexpr (PIPE == PERM_PIPE_FFMA) {
    float x[kProbeChains];
    const float fa = (float)a, fb = (float)b;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = t * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) x[c] = fmaf(x[c], fa, fb);
    }
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
  } else if constexpr (PIPE == PERM_PIPE_FFMA2 || PIPE == PERM_PIPE_ISSUE) {
    float2 x[kProbeChains];
    unsigned u[kProbeChains];
    const float2 fa = make_float2((float)a, (float)a * 0.5f), fb = make_float2((float)b, (float)b * 2.0f);
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = make_float2(t * 1e-3f + c, t * 2e-3f - c), u[c] = t * 7u + c;
    const unsigned ua = (unsigned)t * 0x9E3779B9u, ub = 0x7F4A7C15u;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) {
        x[c] = __ffma2_rn(x[c], fa, fb);
        if constexpr (PIPE == PERM_PIPE_ISSUE)
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(u[c]) : "r"(ua), "r"(ub));
      }
    }
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c].x + x[c].y + (double)u[c];
  } else {
    unsigned x[kProbeChains];
    const unsigned ua = (unsigned)t * 0x9E3779B9u | 1u, ub = 0x7F4A7C15u;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = t * 13u + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) {
        if constexpr (PIPE == PERM_PIPE_IMAD)
          asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(ua), "r"(ub));
        else
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(ua), "r"(ub));
      }
    }
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += (double)x[c];
  }
  sink[(size_t)blockIdx.x * blockDim.x + t] = s;
}

void preload_peak_kernels() {
  load_kernel(k_pipe_probe<PERM_PIPE_DFMA>);
  load_kernel(k_pipe_probe<PERM_PIPE_FFMA>);
  load_kernel(k_pipe_probe<PERM_PIPE_FFMA2>);
  load_kernel(k_pipe_probe<PERM_PIPE_IMAD>);
  load_kernel(k_pipe_probe<PERM_PIPE_ALU>);
  load_kernel(k_pipe_probe<PERM_PIPE_ISSUE>);
}

cudaError_t pipe_probe_launch(int pipe, double* sink, int blocks, int iters, cudaStream_t stream) {
  const double a = 0.999999, b = 1e-7;
  switch (pipe) {
    case PERM_PIPE_DFMA: k_pipe_probe<PERM_PIPE_DFMA><<<blocks, kProbeThreads, 0, stream>>>(sink, iters, a, b); break;
    case PERM_PIPE_FFMA: k_pipe_probe<PERM_PIPE_FFMA><<<blocks, kProbeThreads, 0, stream>>>(sink, iters, a, b); break;
    case PERM_PIPE_FFMA2:
      k_pipe_probe<PERM_PIPE_FFMA2><<<blocks, kProbeThreads, 0, stream>>>(sink, iters, a, b);
      break;
    case PERM_PIPE_IMAD: k_pipe_probe<PERM_PIPE_IMAD><<<blocks, kProbeThreads, 0, stream>>>(sink, iters, a, b); break;
    case PERM_PIPE_ALU: k_pipe_probe<PERM_PIPE_ALU><<<blocks, kProbeThreads, 0, stream>>>(sink, iters, a, b); break;
    case PERM_PIPE_ISSUE:
      k_pipe_probe<PERM_PIPE_ISSUE><<<blocks, kProbeThreads, 0, stream>>>(sink, iters, a, b);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace perm

extern "C" int perm_pipe_peak(int pipe, double* g_per_s) {
  using namespace perm;
  if (!g_per_s) return PERM_ENULL;
  if (pipe < PERM_PIPE_DFMA || pipe > PERM_PIPE_ISSUE) return PERM_EINVAL;
  int count = 0, dev = 0, sms = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) return PERM_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERM_ECUDA;
  const int blocks = sms * 8;
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * blocks * kProbeThreads) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = PERM_OK;
  float best = 1e30f;
  // about 0.02 s per launch for the FP64 probe, ~1 ms for the others
  const int iters = pipe == PERM_PIPE_DFMA ? 4000 : 64000;
  if (pipe_probe_launch(pipe, sink, blocks, iters / 8, nullptr) != cudaSuccess) rc = PERM_ECUDA;
  for (int rep = 0; rep < 5 && rc == PERM_OK; ++rep) {
    cudaEventRecord(e0, nullptr);
    if (pipe_probe_launch(pipe, sink, blocks, iters, nullptr) != cudaSuccess) rc = PERM_ECUDA;
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
  const double per_step = pipe == PERM_PIPE_ISSUE ? 2.0 : 1.0;  // instructions per chain step
  const double ops = (double)blocks * kProbeThreads * kProbeChains * (double)iters * per_step;
  *g_per_s = ops / (best * 1e-3) / 1e9;
  return PERM_OK;
}

extern "C" int perm_fp64_peak(double* gops) { return perm_pipe_peak(PERM_PIPE_DFMA, gops); }

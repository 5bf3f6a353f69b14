// Batched permanents, one block of 128 threads per work item, with the packed
// double-float Gray walk of glynn_walk_xp.cuh (the random-matrix studies of
// Secs. 3-6 need 10^5..10^7 permanents of orders up to ~35).
//
// A persistent grid of these blocks pulls tickets from its own counter; each
// ticket is one (matrix, code chunk) item of an order assigned to this kernel
// (batch_decode).  The block stages that matrix into its shared tables (the
// layout of the single-matrix kernel, sized for the largest order), splits
// the chunk over its threads in congruent ranges, walks, and writes the
// item's double-double partial.  The order is a runtime value; each order
// has its own instantiation of the walk (register arrays need a compile-time
// order), selected per item.  THREADS is the block size (128 or 256: the
// threads that share one item) and MINB the blocks per SM the register
// allocation must allow (2 blocks of 128: up to 255 registers; 3: up to 168;
// 1 block of 256: up to 255), the tuner's choices per order.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "batch_common.cuh"
#include "glynn_walk_xp.cuh"

namespace perm {

constexpr size_t kCtaSmem = XpShape<kBatchNMax, false>::smem_bytes;  // tables of the largest order

template <int N>
__device__ __forceinline__ void cta_item(const double* __restrict__ A, const BatchItemRef& it, float4* smem, int* sG,
                                         dd* sRed, double* __restrict__ partials, int* status, int tile_log) {
  using Shape = XpShape<N, false>;
  constexpr int NP = kPairs<N>;
  float4* sP = smem;
  float4* sM = sP + Shape::table_f4;
  longlong2* sQ = reinterpret_cast<longlong2*>(sM + Shape::table_f4);
  longlong2* sV0 = sQ + (size_t)N * NP * 2;
  const bool bad = xp_stage_df<N>(A, sP, sM, sQ, sV0, sG, status);
  uint64_t r, end;
  range_congruent(it.first, it.count, blockDim.x, threadIdx.x, r, end);
  dd accr{0.0, 0.0}, acci{0.0, 0.0};
  if (!bad) {
    thread_walk_xp_df<N>(sP, sM, sQ, sV0, r, end, tile_log, accr, acci);
    int gs = 0;
    for (int i = 0; i < N; ++i) gs += sG[i];
    const int sc = -N - gs;  // prod_i w_i = prod_i u_i 2^(-N - sum_i G_i)
    accr = dd{scalbn(accr.hi, sc), scalbn(accr.lo, sc)};
    acci = dd{scalbn(acci.hi, sc), scalbn(acci.lo, sc)};
  } else {
    accr = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
    acci = accr;
  }
  __syncthreads();  // every thread is done with the tables
  block_store_to<true>(accr, acci, sRed, partials + it.partial * 4, 0);
  __syncthreads();  // the reduction slots and tables are free for the next item
}

template <int K>
__device__ __forceinline__ void cta_case(const double* __restrict__ A, const BatchItemRef& it, float4* smem, int* sG,
                                         dd* sRed, double* __restrict__ partials, int* status, int tile_log) {
  if constexpr (K <= kBatchNMax) {
    if (it.n == K) {
      cta_item<K>(A, it, smem, sG, sRed, partials, status, tile_log);
      return;
    }
    cta_case<K + 1>(A, it, smem, sG, sRed, partials, status, tile_log);
  }
}

template <int MINB, int THREADS>
__global__ void __launch_bounds__(THREADS, MINB)
    k_batch_cta(const BatchArgs* __restrict__ ba, const int* __restrict__ perm, const __grid_constant__ BatchTable tab,
                int kind, double* __restrict__ partials, unsigned long long* __restrict__ ticket,
                int* __restrict__ status, int tile_log) {
  extern __shared__ __align__(16) float4 csm[];
  __shared__ int sG[kBatchNMax];
  __shared__ dd sRed[2 * (THREADS / 32)];
  __shared__ unsigned long long sTicket;
  const double* const* ptrs = ba->ptrs;
  for (;;) {
    if (threadIdx.x == 0) sTicket = atomicAdd(ticket, 1ull);
    __syncthreads();
    const unsigned long long t = sTicket;
    __syncthreads();  // every thread has its ticket before thread 0 takes the next
    BatchItemRef it;
    if (!batch_decode(tab, kind, perm, t, it)) break;
    cta_case<1>(ptrs[it.matrix], it, csm, sG, sRed, partials, status, tile_log);
  }
}

template <int MINB, int THREADS>
struct CtaKernel {
  static int resident() {
    static std::atomic<int> cached[64];  // per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cached[dev]) return cached[dev];
    if (cudaFuncSetAttribute(k_batch_cta<MINB, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCtaSmem) !=
        cudaSuccess)
      return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_cta<MINB, THREADS>, THREADS, kCtaSmem) !=
        cudaSuccess)
      return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cached[dev] = (per_sm < 1 ? 1 : per_sm) * sms;
    return cached[dev];
  }

  static cudaError_t launch(const BatchArgs* ba, const int* perm, const BatchTable& tab, int kind, double* partials,
                            unsigned long long* ticket, int* status, cudaStream_t s) {
    const int grid = resident();
    if (grid < 1) return cudaErrorInvalidConfiguration;
    k_batch_cta<MINB, THREADS><<<grid, THREADS, kCtaSmem, s>>>(ba, perm, tab, kind, partials, ticket, status,
                                                         pdf_tile_log());
    return cudaGetLastError();
  }
};

}  // namespace perm

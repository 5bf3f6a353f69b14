// Permanents of band matrices (a_ij = 0 for |i - j| > k) by the transfer-
// matrix recursion of App. C ("bandpermanent"): multiply the linear forms
// C_i = sum_j a_ij x_j row by row in formal variables x_1..x_n, with
// x_j^2 = 0, and retire x_{i-k-1} once no later row can touch it.  The work
// is O(n 2^(2k+1) (2k+1)): linear in n for fixed k.
//
// Layout: one CTA per matrix.  Row i's linear form only involves the 2k+1
// variables x_{i-k}..x_{i+k} (the window), so the polynomial is stored densely
// over the 2^(2k+1) subsets of the window, in shared memory (k <= 5: 2048
// complex coefficients, two buffers), of which only the subsets of the one
// size a live monomial can have are formed.  Multiplying by C_i is written in
// gather form, q[T] = sum_{t in T} p[T - t] a_{i, base+t}, so every
// coefficient is produced by one thread in a fixed order (deterministic, no
// atomics).
// Retiring the window's lowest variable keeps the monomials that contain it
// (with the variable set to 1, as in App. C) and shifts the window by one;
// monomials without it can never reach full degree, so they are dropped
// rather than carried (the paper's literal step keeps them, and they vanish
// by the last row; the result is the same).
#include <cuda_runtime.h>

#include <cstdint>

#include "dd.cuh"
#include "glynn_walk.cuh"
#include "perm.h"
#include "perm_internal.h"

namespace perm {

constexpr int kBandThreads = 256;
constexpr int kBandKMax = 5;

// Before row i is multiplied in, every live monomial holds all retired
// variables and min(i, K) window variables; after it, min(i, K) + 1.  Only the
// window subsets of that size are formed (C(2K+1, K+1) of 2^(2K+1) at K = 5);
// entries of other sizes are never read.
template <int K>
__global__ void __launch_bounds__(kBandThreads) k_band(const double* __restrict__ Ag, int n,
                                                       double* __restrict__ out, int* __restrict__ status) {
  constexpr int W = 2 * K + 1;
  constexpr int S = 1 << W;
  extern __shared__ __align__(16) double2 bsmem[];
  double2* p = bsmem;
  double2* q = p + S;
  double2* coef = q + S;
  __shared__ unsigned short ord[S];  // window subsets sorted by size
  __shared__ int off[W + 2];         // subsets of size c are ord[off[c] .. off[c+1])
  __shared__ dd red[2 * (kBandThreads / 32)];
  const double2* A = reinterpret_cast<const double2*>(Ag) + (size_t)blockIdx.x * n * n;

  if (threadIdx.x == 0) {
    int o = 0;
    for (int c = 0; c <= W; ++c) {
      off[c] = o;
      for (int m = 0; m < S; ++m)
        if (__popc(m) == c) ord[o++] = (unsigned short)m;
    }
    off[W + 1] = o;
  }
  for (int m = threadIdx.x; m < S; m += kBandThreads) p[m] = make_double2(m == 0 ? 1.0 : 0.0, 0.0);
  __syncthreads();
  int bad = 0;
  int deg = 0;  // size of the live subsets after the current row
  for (int i = 0; i < n; ++i) {
    const int base = i - K;  // variable index of window bit 0
    deg = (i < K ? i : K) + 1;
    if (threadIdx.x < W) {
      const int j = base + (int)threadIdx.x;
      double2 a = make_double2(0.0, 0.0);
      if (j >= 0 && j < n) {
        a = A[(size_t)i * n + j];
        bad |= (not_finite(a.x) || not_finite(a.y)) ? 1 : 0;
      }
      coef[threadIdx.x] = a;
    }
    __syncthreads();
    // q = p * C_i with x_j^2 = 0, on the subsets of size deg
    for (int t2 = off[deg] + threadIdx.x; t2 < off[deg + 1]; t2 += kBandThreads) {
      const int T = ord[t2];
      double qr = 0.0, qi = 0.0;
#pragma unroll
      for (int t = 0; t < W; ++t) {
        if ((T >> t) & 1) {
          const double2 c = coef[t];
          const double2 v = p[T & ~(1 << t)];
          qr = fma(v.x, c.x, qr);
          qr = fma(-v.y, c.y, qr);
          qi = fma(v.x, c.y, qi);
          qi = fma(v.y, c.x, qi);
        }
      }
      q[T] = make_double2(qr, qi);
    }
    __syncthreads();
    if (i + 1 < n) {
      // retire variable `base` (window bit 0) and shift the window by one;
      // the new top bit (x_{i+1+K}) has not been multiplied in yet
      for (int Sn = threadIdx.x; Sn < S; Sn += kBandThreads) {
        double2 v = make_double2(0.0, 0.0);
        if (!((Sn >> (W - 1)) & 1)) {
          const int T = base >= 0 ? ((Sn << 1) | 1) : (Sn << 1);
          if (__popc(T) == deg) v = q[T];
        }
        p[Sn] = v;
      }
      __syncthreads();
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, (int)kStatusNonFinite);
  // all x := 1: sum of the coefficients (only the full monomial survives)
  dd sr{0.0, 0.0}, si{0.0, 0.0};
  for (int t2 = off[deg] + threadIdx.x; t2 < off[deg + 1]; t2 += kBandThreads) {
    const int T = ord[t2];
    sr = dd_add_d(sr, q[T].x);
    si = dd_add_d(si, q[T].y);
  }
  sr = dd_warp_sum_exact(sr);
  si = dd_warp_sum_exact(si);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[2 * warp] = sr;
    red[2 * warp + 1] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    dd tr = red[0], ti = red[1];
    for (int w = 1; w < kBandThreads / 32; ++w) {
      tr = dd_add(tr, red[2 * w]);
      ti = dd_add(ti, red[2 * w + 1]);
    }
    out[2 * (size_t)blockIdx.x] = __dadd_rn(tr.hi, tr.lo);
    out[2 * (size_t)blockIdx.x + 1] = __dadd_rn(ti.hi, ti.lo);
  }
}

template <int LO, int HI>
cudaError_t band_dispatch(int k, const double* A, int n, int count, double* out, int* status, cudaStream_t s) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    if (k == LO) {
      constexpr size_t smem = (size_t)(2 * (1 << (2 * LO + 1)) + 2 * LO + 1) * sizeof(double2);
      if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_band<LO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      k_band<LO><<<count, kBandThreads, smem, s>>>(A, n, out, status);
      return cudaGetLastError();
    }
    return band_dispatch<LO + 1, HI>(k, A, n, count, out, status, s);
  }
}

template <int LO, int HI>
void band_preload() {
  if constexpr (LO <= HI) {
    load_kernel(k_band<LO>);
    band_preload<LO + 1, HI>();
  }
}

void preload_band_kernels() { band_preload<0, kBandKMax>(); }

}  // namespace perm

namespace {

bool device_ptr_band(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int perm_c128_band(const double* A, int n, int k, int count, double* out, void* stream) {
  using namespace perm;
  TraceRange trace("perm_c128_band");
  if (n < 1 || n > 65535 || k < 0 || k > kBandKMax || count < 1 || count > (1 << 30)) return PERM_EINVAL;
  // count * n * n complex entries must be addressable: at most 2^44 (256 TiB),
  // far beyond any device, so the byte counts below cannot wrap
  if ((double)count * (double)n * (double)n > 17592186044416.0) return PERM_EINVAL;
  if (!A || !out) return PERM_ENULL;
  int ndev = 0, dev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) return PERM_ECUDA;
  ensure_kernels_loaded();
  int* status = nullptr;
  if (device_status_word(dev, &status) != 0) return PERM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytesA = (size_t)count * n * n * 16;
  const size_t bytesO = (size_t)count * 16;
  const bool a_dev = device_ptr_band(A), o_dev = device_ptr_band(out);
  const size_t szA = a_dev ? 0 : ((bytesA + 255) & ~(size_t)255);
  const size_t szO = o_dev ? 0 : ((bytesO + 255) & ~(size_t)255);
  char* base = nullptr;
  cudaError_t e = cudaSuccess;
  if (szA + szO) {
    e = cudaMallocAsync((void**)&base, szA + szO, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? PERM_ENOMEM : PERM_ECUDA;
    }
  }
  const double* dA = A;
  if (!a_dev) {
    e = cudaMemcpyAsync(base, A, bytesA, cudaMemcpyHostToDevice, s);
    dA = (const double*)base;
  }
  double* dOut = o_dev ? out : (double*)(base + szA);
  if (e == cudaSuccess) e = band_dispatch<0, kBandKMax>(k, dA, n, count, dOut, status, s);
  if (e == cudaSuccess && !o_dev) e = cudaMemcpyAsync(out, dOut, bytesO, cudaMemcpyDeviceToHost, s);
  if (base) cudaFreeAsync(base, s);
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

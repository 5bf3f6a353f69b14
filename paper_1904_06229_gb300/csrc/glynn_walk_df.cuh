// Gray-code walk with double-float arithmetic on the FP32 pipe (the same sum
// as glynn_walk.cuh: Sec. 2.A, App. A).
//
// GB300 issues FP32 FMAs 64x faster than FP64 ones.  This walk keeps each row
// sum as an unevaluated pair of floats (hi + lo, about 48 significant bits:
// Dekker's double-length representation) and forms the products with
// error-free transformations built from FMA (the exact product error
// fma(a, b, -a*b) and Knuth's TwoSum).  Row sums and column steps are scaled
// by 2^-62 per row (|u_i| < 1); the row scales multiply the whole sum once.
//
// Accuracy: a double-float addition or multiplication is accurate to about
// 2^-47 relative, so the row sums drift by about sqrt(steps) 2^-48; every run
// of 128 codes re-seeds them from exact int64 fixed-point row sums (the same
// quantisation as the fixed-point walk), and the partial products (four
// interleaved chains) are renormalised by powers of two every 8 factors so
// they never leave the FP32 range.  Terms are rebuilt as doubles with integer
// bit operations and summed like the other walks (FP64 run sums folded into
// double-double).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include <cstdint>

#include "dd.cuh"
#include "glynn_walk.cuh"
#include "glynn_walk_fx.cuh"
#include "perm_internal.h"

namespace perm {

constexpr int kDfRunLog = 7;
constexpr uint64_t kDfRun = 1ull << kDfRunLog;

// Knuth's TwoSum on floats: s + e == a + b exactly.
__device__ __forceinline__ void f_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// double-float addition (both halves through TwoSum, then renormalised)
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  f_two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// a*b - c*d for double-floats.  The result is left as TwoSum's (s, e) plus
// the products' low parts: |l| stays within a few units of the last place of
// h, which the next product's FMAs take as it is (the pair is renormalised
// only where it is stored: in the row sums, by df_add).
__device__ __forceinline__ void df_mul_sub(float ah, float al, float bh, float bl, float ch, float cl, float dh,
                                           float dl, float& h, float& l) {
  const float p1 = __fmul_rn(ah, bh);
  float e1 = __fmaf_rn(ah, bh, -p1);
  e1 = __fmaf_rn(ah, bl, e1);
  e1 = __fmaf_rn(al, bh, e1);
  const float p2 = __fmul_rn(ch, dh);
  float e2 = __fmaf_rn(ch, dh, -p2);
  e2 = __fmaf_rn(ch, dl, e2);
  e2 = __fmaf_rn(cl, dh, e2);
  float s, e;
  f_two_sum(p1, -p2, s, e);
  h = s;
  l = __fadd_rn(e, __fsub_rn(e1, e2));
}

// a*b + c*d for double-floats, result renormalised.
__device__ __forceinline__ void df_mul_add(float ah, float al, float bh, float bl, float ch, float cl, float dh,
                                           float dl, float& h, float& l) {
  df_mul_sub(ah, al, bh, bl, -ch, -cl, dh, dl, h, l);
}

struct cdf {
  float rh, rl, ih, il;
};

__device__ __forceinline__ cdf cdf_mul(const cdf& a, const cdf& b) {
  cdf r;
  df_mul_sub(a.rh, a.rl, b.rh, b.rl, a.ih, a.il, b.ih, b.il, r.rh, r.rl);
  df_mul_add(a.rh, a.rl, b.ih, b.il, a.ih, a.il, b.rh, b.rl, r.ih, r.il);
  return r;
}

// Scale a complex double-float by a power of two so its larger high part lies
// in [1, 2); the exponent removed is added to E.  Zero stays zero.
__device__ __forceinline__ void cdf_renorm(cdf& a, int& E) {
  const int er = (__float_as_int(a.rh) >> 23) & 0xff;
  const int ei = (__float_as_int(a.ih) >> 23) & 0xff;
  const int em = max(er, ei);
  if (em == 0) return;
  const int e = em - 127;
  const float sc = __int_as_float((127 - e) << 23);  // 2^-e, a normal float for |e| <= 126
  a.rh *= sc;
  a.rl *= sc;
  a.ih *= sc;
  a.il *= sc;
  E += e;
}

// Split a double into a double-float (h = nearest float, l = nearest float of the rest).
__device__ __forceinline__ void split_double(double d, float& h, float& l) {
  h = __double2float_rn(d);
  l = __double2float_rn(d - (double)h);
}

// Product of the N row sums in four interleaved chains (rows i = c mod 4),
// each renormalised by a power of two every 8 factors, then combined.
template <int N>
__device__ __forceinline__ void df_product(const cdf (&u)[N], double& pr, double& pi) {
  constexpr int NC = N < 4 ? N : 4;
  cdf p[NC];
  int E[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) p[c] = u[c], E[c] = 0;
#pragma unroll
  for (int i = NC; i < N; ++i) {
    const int c = i % NC;
    p[c] = cdf_mul(p[c], u[i]);
    if ((i / NC) % 8 == 7) cdf_renorm(p[c], E[c]);
  }
  int Et = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) cdf_renorm(p[c], E[c]), Et += E[c];
  if constexpr (NC >= 2) p[0] = cdf_mul(p[0], p[1]);
  if constexpr (NC >= 4) {
    p[2] = cdf_mul(p[2], p[3]);
    p[0] = cdf_mul(p[0], p[2]);
  } else if constexpr (NC == 3) {
    p[0] = cdf_mul(p[0], p[2]);
  }
  pr = f32_times_pow2(p[0].rh, Et) + f32_times_pow2(p[0].rl, Et);
  pi = f32_times_pow2(p[0].ih, Et) + f32_times_pow2(p[0].il, Et);
}

template <int N>
struct DfShape {
  // +2A int64 table (column-major, for exact re-seeds), +2A and -2A double-float
  // tables (float4 per entry), v0 (int64), per-row exponents, reduction slots
  static constexpr size_t smem_bytes = (size_t)N * N * sizeof(longlong2) + 2 * (size_t)N * N * sizeof(float4) +
                                       (size_t)N * sizeof(longlong2) + 2 * N * sizeof(int) + 8 * sizeof(dd) + 16;
};

template <int N>
__global__ void __launch_bounds__(kWalkThreads) k_walk_df(const double* __restrict__ A, uint64_t first, uint64_t count,
                                                          double* __restrict__ partials, int accumulate,
                                                          int* __restrict__ status) {
  extern __shared__ __align__(16) long long dsm[];
  longlong2* sP = reinterpret_cast<longlong2*>(dsm);  // +2A_ij (int64), [j * N + i]
  float4* sDp = reinterpret_cast<float4*>(sP + N * N);  // +2A_ij 2^-62 as (rh, rl, ih, il)
  float4* sDm = sDp + N * N;                            // -2A_ij 2^-62
  longlong2* sV0 = reinterpret_cast<longlong2*>(sDm + N * N);
  int* sF = reinterpret_cast<int*>(sV0 + N);
  int* sEb = sF + N;
  dd* sRed = reinterpret_cast<dd*>(dsm);  // reused after the walk

  // ---- stage: per-row scales and exact tables as in the fixed-point walk
  int bad = 0;
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
    double mx = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      double s = 0.0;
      for (int j = 0; j < N; ++j) {
        const double v = A[((size_t)i * N + j) * 2 + c];
        bad |= not_finite(v) ? 1 : 0;
        s += fabs(v);
      }
      mx = fmax(mx, s);
    }
    int F = 0;
    if (mx > 0.0 && !bad) {
      const int ex = dexp_of(mx);
      F = ex == 0 ? 61 + 1022 : 61 - (ex - 1023);
    }
    sF[i] = F;
    sEb[i] = 1024;  // fx_to_double(v, 1024) = v 2^-62
  }
  const bool any_bad = __syncthreads_or(bad) != 0;
  if (any_bad && threadIdx.x == 0) atomicOr(status, (int)kStatusNonFinite);
  if (!any_bad) {
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int i = idx / N, j = idx - i * N;
      const int F = sF[i];
      const long long qr = 2 * __double2ll_rn(scalbn(A[(size_t)idx * 2], F));
      const long long qi = 2 * __double2ll_rn(scalbn(A[(size_t)idx * 2 + 1], F));
      sP[j * N + i] = make_longlong2(qr, qi);
      float4 d;
      split_double(fx_to_double(qr, 1024), d.x, d.y);
      split_double(fx_to_double(qi, 1024), d.z, d.w);
      sDp[j * N + i] = d;
      sDm[j * N + i] = make_float4(-d.x, -d.y, -d.z, -d.w);
    }
  }
  __syncthreads();
  if (threadIdx.x < N && !any_bad) {
    const int i = threadIdx.x;
    long long sr = sP[(N - 1) * N + i].x, si = sP[(N - 1) * N + i].y;
    for (int j = 0; j < N - 1; ++j) sr -= sP[j * N + i].x, si -= sP[j * N + i].y;
    sV0[i] = make_longlong2(sr / 2, si / 2);
  }
  __syncthreads();
  // w_i = v_i 2^(-F_i - 1) = u_i 2^(61 - F_i) with u_i = v_i 2^-62
  int Esum = 0;
  for (int i = 0; i < N; ++i) Esum += 61 - sF[i];

  uint64_t r, end;
  thread_range(first, count, r, end);
  dd accr{0.0, 0.0}, acci{0.0, 0.0};
  if (any_bad) {
    accr = acci = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
  } else {
    cdf u[N];
    while (r < end) {
      const uint64_t run_end = min(end, (r | (kDfRun - 1)) + 1);
      {
        // exact re-seed: v = v0 + sum_{j<n, x_j=1} 2A_ij (int64), then u = v 2^-62
        const uint64_t x = r ^ (r >> 1);
        float4 seed[N];
#pragma unroll 1
        for (int i = 0; i < N; ++i) {
          long long sr = sV0[i].x, si = sV0[i].y;
#pragma unroll 1
          for (int j = 0; j < N - 1; ++j)
            if ((x >> j) & 1ull) sr += sP[j * N + i].x, si += sP[j * N + i].y;
          float4 d;
          split_double(fx_to_double(sr, 1024), d.x, d.y);
          split_double(fx_to_double(si, 1024), d.z, d.w);
          seed[i] = d;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) u[i] = cdf{seed[i].x, seed[i].y, seed[i].z, seed[i].w};
      }
      double sr = 0.0, si = 0.0;
      uint32_t odd = (uint32_t)(r & 1ull);
      for (; r < run_end; ++r) {
        double pr, pi;
        df_product<N>(u, pr, pi);
        const double sg = pm_one(odd);
        odd ^= 1u;
        sr = fma(sg, pr, sr);
        si = fma(sg, pi, si);
        int j;
        uint32_t neg;
        gray_step(r, j, neg);
        const float4* col = (neg ? sDm : sDp) + j * N;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const float4 c = col[i];
          df_add(u[i].rh, u[i].rl, c.x, c.y, u[i].rh, u[i].rl);
          df_add(u[i].ih, u[i].il, c.z, c.w, u[i].ih, u[i].il);
        }
      }
      accr = dd_add_d(accr, sr);
      acci = dd_add_d(acci, si);
    }
    // the row scales, once: prod_i 2^(61 - F_i)
    accr = dd{scalbn(accr.hi, Esum), scalbn(accr.lo, Esum)};
    acci = dd{scalbn(acci.hi, Esum), scalbn(acci.lo, Esum)};
  }
  __syncthreads();
  block_store<true>(accr, acci, sRed, partials, accumulate);
}

template <int N>
struct DfKernel {
  static constexpr size_t smem = DfShape<N>::smem_bytes;

  static cudaError_t prepare(int& resident) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::atomic<int> cached[64];  // per device; filled once, read from any host thread
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (cached[dev] > 0) {
      resident = cached[dev];
      return cudaSuccess;
    }
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(k_walk_df<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_df<N>, kWalkThreads, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    cached[dev] = per_sm * sms;
    resident = cached[dev];
    return cudaSuccess;
  }

  static int resident_blocks() {
    int r = 0;
    return prepare(r) == cudaSuccess ? r : 0;
  }

  static cudaError_t launch(const WalkArgs& a) {
    int resident = 0;
    cudaError_t e = prepare(resident);
    if (e != cudaSuccess) return e;
    k_walk_df<N><<<a.blocks, kWalkThreads, smem, a.stream>>>(a.A, a.first, a.count, a.partials, a.accumulate,
                                                              a.status);
    return cudaGetLastError();
  }
};

template <int LO, int HI>
cudaError_t df_dispatch(const WalkArgs& a) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    if (a.n == LO) return DfKernel<LO>::launch(a);
    return df_dispatch<LO + 1, HI>(a);
  }
}

template <int LO, int HI>
int df_blocks_dispatch(int n) {
  if constexpr (LO > HI) {
    return 0;
  } else {
    if (n == LO) return DfKernel<LO>::resident_blocks();
    return df_blocks_dispatch<LO + 1, HI>(n);
  }
}

}  // namespace perm

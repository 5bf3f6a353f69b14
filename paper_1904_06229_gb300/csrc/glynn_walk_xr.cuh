// Real matrices: the packed double-float Gray walk of glynn_walk_xp.cuh with
// one component per row (the same sum: Sec. 2.A, App. A).
//
// Rows 2k and 2k+1 again share the two lanes of every packed register pair;
// a real row pair is one double-float pair (h, l), so the walk keeps 4
// registers per row pair instead of 8, a step's update is one double-float
// add (11 packed operations) per pair, and a product step is an exact FP32
// product by FMA with its two cross terms (4 packed operations, low part left
// unrenormalised).  Six chains in three packed chain pairs (measured against
// two, four and five pairs at n = 32, 36, 40: three is 4-6 % faster than four
// at every order; two wins only at n = 32), power-of-two renormalisation every
// eight factors and at the end; the lanes are joined by one scalar
// double-float product and the term is rebuilt as FP64 like the complex
// walk's.  Re-seeds from exact int64 rows every 2^tile_log codes as
// in the complex walk.
#pragma once

#include "glynn_walk_xp.cuh"

namespace perm {

template <int N>
struct XrShape {
  static constexpr int NP = kPairs<N>;
  // +c and -c tables: [column j < N][pair k] float4 (h.x, h.y, l.x, l.y)
  static constexpr size_t table_f4 = (size_t)N * NP;
  // int64 columns [k][j] longlong2 (row 2k, row 2k+1), then seeds [k]
  static constexpr size_t seed_bytes = ((size_t)N * NP + NP) * sizeof(longlong2);
  static constexpr size_t smem_bytes = 2 * table_f4 * sizeof(float4) + seed_bytes + 8 * sizeof(dd) + 16;
};

constexpr int kXrChainPairs = 3;

// Two real double-float numbers side by side (lanes .x and .y).
struct P2 {
  float2 h, l;
};

// a * b: exact product of the high parts by FMA plus the two cross terms; the
// low part is left within a few units of the last place of the high part.
__device__ __forceinline__ P2 p2_mul(const P2& a, const P2& b) {
  P2 r;
  r.h = f2mul(a.h, b.h);
  float2 e = f2fma(a.h, b.h, f2neg(r.h));
  e = f2fma(a.h, b.l, e);
  r.l = f2fma(a.l, b.h, e);
  return r;
}

// Scale each lane by a power of two so that its high part lies in [1, 2); a
// zero (or subnormal) lane is left as it is.
__device__ __forceinline__ void p2_renorm(P2& a, int& ex, int& ey) {
  int mx = (__float_as_int(a.h.x) >> 23) & 0xff, my = (__float_as_int(a.h.y) >> 23) & 0xff;
  mx = mx ? mx : 127;
  my = my ? my : 127;
  const float2 sc = make_float2(__int_as_float((254 - mx) << 23), __int_as_float((254 - my) << 23));
  a.h = f2mul(a.h, sc);
  a.l = f2mul(a.l, sc);
  ex += mx - 127;
  ey += my - 127;
}

// Product of the N row sums as a double-float (zh + zl) times 2^E.
template <int N>
__device__ __forceinline__ void xr_product(const P2 (&v)[kPairs<N>], float& zh, float& zl, int& E) {
  constexpr int NP = kPairs<N>;
  constexpr int CP = NP >= kXrChainPairs ? kXrChainPairs : NP;
  P2 c[CP];
  int ex[CP], ey[CP], len[CP];
#pragma unroll
  for (int q = 0; q < CP; ++q) c[q] = v[q], ex[q] = 0, ey[q] = 0, len[q] = 1;
#pragma unroll
  for (int k = CP; k < NP; ++k) {
    const int q = k % CP;
    c[q] = p2_mul(c[q], v[k]);
    if (++len[q] % kXpRenormEvery == 0 && k + CP < NP) p2_renorm(c[q], ex[q], ey[q]);
  }
#pragma unroll
  for (int q = 0; q < CP; ++q) p2_renorm(c[q], ex[q], ey[q]);
#pragma unroll
  for (int q = 1; q < CP; ++q) {
    c[0] = p2_mul(c[0], c[q]);
    ex[0] += ex[q];
    ey[0] += ey[q];
  }
  const float ph = __fmul_rn(c[0].h.x, c[0].h.y);
  float pe = __fmaf_rn(c[0].h.x, c[0].h.y, -ph);
  pe = __fmaf_rn(c[0].h.x, c[0].l.y, pe);
  pe = __fmaf_rn(c[0].l.x, c[0].h.y, pe);
  zh = ph;
  zl = pe;
  E = ex[0] + ey[0];
}

// Stage: Q_ij = rint(a_ij 2^(G_i + 61)); the int64 columns 2 Q_ij (sQ, [k][j],
// lanes = rows 2k, 2k+1) and seeds v0_i = Q_in - sum_{j<n} Q_ij (sV0, [k]);
// the +c / -c tables of their double-float roundings.  Returns whether any
// entry is non-finite.
template <int N>
__device__ __forceinline__ bool xr_stage_df(const double* __restrict__ A, float4* sP, float4* sM, longlong2* sQ,
                                            longlong2* sV0, int* sG, int* status) {
  constexpr int NP = kPairs<N>;
  if (xp_row_scales<N, 1>(A, sG, status)) return true;
  float* fP = reinterpret_cast<float*>(sP);
  float* fM = reinterpret_cast<float*>(sM);
  long long* q64 = reinterpret_cast<long long*>(sQ);
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const int k = i >> 1, lane = i & 1;
    float h = 0.f, l = 0.f;
    long long q2 = 0;
    const long long q = __double2ll_rn(scalbn(A[idx], sG[i] + kPdfGrid));
    if (j < N - 1) {
      q2 = 2 * q;
      pdf_split(q2, h, l);
    }
    const size_t base = ((size_t)j * NP + k) * 4;
    fP[base + lane] = h;
    fP[base + 2 + lane] = l;
    fM[base + lane] = -h;
    fM[base + 2 + lane] = -l;
    q64[((size_t)k * N + j) * 2 + lane] = q2;
    if (j == N - 1) reinterpret_cast<long long*>(sV0)[k * 2 + lane] = q;  // Q_in, completed below
  }
  long long* v64 = reinterpret_cast<long long*>(sV0);
  if (N & 1) {
    // the missing row of an odd order: constant 1 (seed 2^61, columns zero)
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const size_t base = ((size_t)j * NP + (NP - 1)) * 4;
      fP[base + 1] = 0.f, fP[base + 3] = 0.f;
      fM[base + 1] = 0.f, fM[base + 3] = 0.f;
      q64[((size_t)(NP - 1) * N + j) * 2 + 1] = 0;
    }
    if (threadIdx.x == 0) v64[(NP - 1) * 2 + 1] = 1ll << kPdfGrid;
  }
  __syncthreads();
  // seeds v0_i = Q_in - sum_{j<n} Q_ij from the int64 table (exact integer sums)
  if (threadIdx.x < N) {
    const int i = threadIdx.x, k = i >> 1, lane = i & 1;
    long long s = v64[k * 2 + lane];
    for (int j = 0; j < N - 1; ++j) s -= q64[((size_t)k * N + j) * 2 + lane] >> 1;
    v64[k * 2 + lane] = s;
  }
  __syncthreads();
  return false;
}

// Re-seed every row pair from its exact int64 value at code r.
template <int N>
__device__ __forceinline__ void xr_seed(P2 (&v)[kPairs<N>], const longlong2* __restrict__ sQ,
                                        const longlong2* __restrict__ sV0, uint64_t r) {
  constexpr int NP = kPairs<N>;
  const uint64_t x0 = r ^ (r >> 1);
  P2 seed[NP];
#pragma unroll 1
  for (int k = 0; k < NP; ++k) {
    longlong2 a = sV0[k];
    uint64_t x = x0;
#pragma unroll 1
    while (x) {
      const int j = __ffsll((long long)x) - 1;
      x &= x - 1;
      const longlong2 q = sQ[(size_t)k * N + j];
      a.x += q.x;
      a.y += q.y;
    }
    P2 t;
    pdf_split(a.x, t.h.x, t.l.x);
    pdf_split(a.y, t.h.y, t.l.y);
    seed[k] = t;
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) v[k] = seed[k];
}

template <int N>
__device__ __forceinline__ void thread_walk_xr_df(const float4* __restrict__ sP, const float4* __restrict__ sM,
                                                  const longlong2* __restrict__ sQ,
                                                  const longlong2* __restrict__ sV0, uint64_t r, const uint64_t end,
                                                  int tile_log, dd& acc) {
  constexpr int NP = kPairs<N>;
  P2 v[NP];
  while (r < end) {
    const uint64_t tile_end = min(end, r + (uint64_t)(1ull << tile_log));
    xr_seed<N>(v, sQ, sV0, r);
    double s = 0.0;
    uint32_t odd = (uint32_t)(r & 1ull);
    for (; r < tile_end; ++r) {
      float zh, zl;
      int E;
      xr_product<N>(v, zh, zl, E);
      s += f32_scaled_f64(zh, E, odd);
      s += f32_scaled_f64(zl, E, odd);
      odd ^= 1u;
      int j;
      uint32_t neg;
      gray_step(r, j, neg);
      const float4* col = (neg ? sM : sP) + (size_t)j * NP;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const float4 c = col[k];
        df2_add(v[k].h, v[k].l, make_float2(c.x, c.y), make_float2(c.z, c.w));
      }
    }
    acc = dd_add_d(acc, s);
  }
}

template <int N>
__global__ void __launch_bounds__(kWalkThreads) k_walk_xr(const double* __restrict__ A, uint64_t first,
                                                          uint64_t count, double* __restrict__ partials,
                                                          int accumulate, int* __restrict__ status, int tile_log) {
  using Shape = XrShape<N>;
  constexpr int NP = kPairs<N>;
  extern __shared__ __align__(16) float4 rsm[];
  float4* sP = rsm;
  float4* sM = sP + Shape::table_f4;
  longlong2* sQ = reinterpret_cast<longlong2*>(sM + Shape::table_f4);
  longlong2* sV0 = sQ + (size_t)N * NP;
  __shared__ int sG[N];
  dd* sRed = reinterpret_cast<dd*>(sV0 + NP);
  const bool bad = xr_stage_df<N>(A, sP, sM, sQ, sV0, sG, status);
  uint64_t r, end;
  thread_range_congruent(first, count, r, end);
  dd acc{0.0, 0.0};
  if (!bad) {
    thread_walk_xr_df<N>(sP, sM, sQ, sV0, r, end, tile_log, acc);
    int gs = 0;
    for (int i = 0; i < N; ++i) gs += sG[i];
    const int sc = -N - gs;  // prod_i w_i = prod_i u_i 2^(-N - sum_i G_i)
    acc = dd{scalbn(acc.hi, sc), scalbn(acc.lo, sc)};
  } else {
    acc = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
  }
  __syncthreads();
  block_store<false>(acc, acc, sRed, partials, accumulate);
}

template <int N>
struct XrKernel {
  static constexpr size_t smem = XrShape<N>::smem_bytes;

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
      e = cudaFuncSetAttribute(k_walk_xr<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_xr<N>, kWalkThreads, smem);
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
    k_walk_xr<N><<<a.blocks, kWalkThreads, smem, a.stream>>>(a.A, a.first, a.count, a.partials, a.accumulate,
                                                              a.status, pdf_tile_log());
    return cudaGetLastError();
  }
};

template <int LO, int HI>
cudaError_t xr_dispatch(const WalkArgs& a) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    if (a.n == LO) return XrKernel<LO>::launch(a);
    return xr_dispatch<LO + 1, HI>(a);
  }
}

template <int LO, int HI>
int xr_blocks_dispatch(int n) {
  if constexpr (LO > HI) {
    return 0;
  } else {
    if (n == LO) return XrKernel<LO>::resident_blocks();
    return xr_blocks_dispatch<LO + 1, HI>(n);
  }
}

}  // namespace perm

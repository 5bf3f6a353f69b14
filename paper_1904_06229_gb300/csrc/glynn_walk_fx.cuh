// Gray-code walk with exact fixed-point row sums (the same sum as
// glynn_walk.cuh: Sec. 2.A, App. A).
//
// Each row i of A is scaled by its own power of two 2^F_i (chosen so that
// sum_j |a_ij| 2^F_i < 2^62) and rounded once to int64: A_ij = rint(a_ij 2^F_i).
// The row sums are then carried in Glynn's form v_i = 2 w_i = sum_{j<n} e_j
// A_ij + A_{i,n} (e_j = +-1) as exact int64: the per-code update is an
// integer add of +-2 A_ij, so the row sums never drift and need no re-seeding;
// the only rounding in a row sum is the one-time rounding of A to 2^-F_i,
// at least as fine as a 53-bit double of the row's largest sum.
//
// Per code, for complex A the first kIxRows<N> (about 0.85 n) of the v_i are
// multiplied straight from their integers in 64-bit integer block floating
// point (see ix_product below); each remaining v_i is turned into the double
// w_i = v_i 2^(-F_i - 1) with integer bit operations (sign, count of leading
// zeros, shift, exponent field; truncated to 53 bits) and multiplied in
// FP64, and the signed accumulation runs in FP64 as in the floating-point
// walk (in the FP32-product mode, v_i is split straight into an FP32
// significand and an integer exponent).
//
// GB300 note: DFMA issues at 1/64 of the FP32 rate on this part while the
// integer pipes run at half the FP32 rate, so the 2n row-update adds per code
// run on the integer pipes, and so does most of the product: the FP64 pipe
// keeps 4 (n - kIxRows) + 4 operations per complex code (28 at n = 40,
// against 6n - 2 = 238 for FP64 row sums and products).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include <cstdint>

#include "dd.cuh"
#include "glynn_walk.cuh"
#include "perm_internal.h"

namespace perm {

template <int N, bool CPLX>
struct FxShape {
  static constexpr int E = CPLX ? 2 : 1;
  // Column stride of the tables: an odd number of entries, so that the columns
  // that the threads of a warp read at once (each at its own Gray code) start
  // in different shared-memory banks.
  static constexpr int S = N | 1;
  // +2A and -2A tables (int64, column-major), v0 (int64), two per-row int
  // arrays (exponent biases sEb, scales sF); the kernel takes its pointers from
  // these offsets.  The dd reduction slots reuse the tables after the walk.
  static constexpr size_t table_bytes = (size_t)N * S * E * sizeof(long long);
  static constexpr size_t v0_off = 2 * table_bytes;
  static constexpr size_t eb_off = v0_off + (size_t)N * E * sizeof(long long);
  static constexpr size_t f_off = eb_off + (size_t)N * sizeof(int);
  static constexpr size_t smem_bytes = f_off + (size_t)N * sizeof(int) + 8 * sizeof(dd) + 16;
};

// Double with value v * 2^(eb - 1086) (eb = 1086 - scale exponent), from the
// bits of v only: |v| normalised by its leading-zero count, 52 fraction bits
// kept, exponent field from the leading-zero count.  RN = false truncates
// (the Gray walks: a truncation bias scales every term alike and does not
// meet the sum's cancellation); RN = true rounds to nearest (half-way cases
// away from zero; used by the un-halved sums, whose terms are all large).
// 0 for v == 0 and for results below the normal range.
template <bool RN = false>
__device__ __forceinline__ double fx_to_double(long long v, int eb) {
  const unsigned long long s = (unsigned long long)(v >> 63);
  const unsigned long long m = ((unsigned long long)v ^ s) - s;
  const int lz = __clzll((long long)m);
  unsigned long long mn = m << (lz & 63);
  int up = 0;
  if constexpr (RN) {
    const unsigned long long rn = mn + 0x400ull;  // + half a unit of the 53rd bit
    up = rn < mn ? 1 : 0;                         // rounding carried past bit 63
    mn = rn;
  }
  const uint32_t hi = (uint32_t)(mn >> 32), lo = (uint32_t)mn;
  const int be = eb - lz + up;  // biased exponent of the result
  const uint32_t dhi = ((uint32_t)s & 0x80000000u) | ((uint32_t)be << 20) | ((hi >> 11) & 0xFFFFFu);
  const uint32_t dlo = (hi << 21) | (lo >> 11);
  return (m == 0 || be <= 0) ? 0.0 : __hiloint2double((int)dhi, (int)dlo);
}

// FP32 significand of v scaled by 2^-(63 - lzref), i.e. relative to a number
// whose leading one sits at bit 63 - lzref; 0 when v == 0 or far below.
__device__ __forceinline__ float fx_to_f32(long long v, int lzref) {
  const unsigned long long s = (unsigned long long)(v >> 63);
  const unsigned long long m = ((unsigned long long)v ^ s) - s;
  const int lz = __clzll((long long)m);
  const unsigned long long mn = m << (lz & 63);
  const int fexp = 127 + lzref - lz;
  uint32_t bits = ((uint32_t)s & 0x80000000u) | ((uint32_t)fexp << 23) | ((uint32_t)(mn >> 40) & 0x7FFFFFu);
  bits += (uint32_t)(mn >> 39) & 1u;  // round half up on the magnitude (a carry moves into the exponent)
  return (m == 0 || fexp <= 0) ? 0.0f : __int_as_float((int)bits);
}

template <int N, bool CPLX, int MODE, bool RN = false>
struct FxProduct;

// ---- integer block floating point for part of the complex product ----
// The FP64 pipe bounds the walk (four DFMAs per factor) while the integer
// pipes have room, so the product of the first kIxRows<N> row sums (about
// 0.85 n, the best of the splits measured at n = 40; at least two rows stay
// in FP64) is formed from their exact int64 values in 64-bit integer block
// floating point: a
// complex number (X + iY) 2^e with int64 X, Y and max(|X|, |Y|) brought to
// [2^61, 2^62] by a left shift; each factor is shifted into the same range,
// the complex product is formed from 32-bit pieces (each step errs by under
// 2^-56 of the result, finer than FP64 rounding), and the result is
// renormalised.  The block enters the FP64 chains once per term as one
// complex double.
template <int N>
constexpr int kIxRows = N >= 8 ? ((N * 17) / 20 < N - 2 ? (N * 17) / 20 : N - 2) : 0;

__device__ __forceinline__ int ix_shift(long long x, long long y) {
  const unsigned long long m = (unsigned long long)(x ^ (x >> 63)) | (unsigned long long)(y ^ (y >> 63));
  return max(__clzll((long long)m) - 2, 0);
}

__device__ __forceinline__ long long ix_shl(long long x, int k) { return (long long)((unsigned long long)x << k); }

// One step of a block: (X + iY) 2^e times (a + ib) 2^f, both normalised.
// Each 64-bit operand is taken as a signed high word h (|h| <= 2^30) and a
// 30-bit low part l (its low 32 bits without the last two), so that
// x a 2^-64 = x_h a_h + (x_h a_l + x_l a_h) 2^-30 up to the dropped low-by-low
// and last-two-bit terms (under 4 units of a result of at least 2^56): twelve
// widening 32-bit multiply-adds instead of four 64 x 64-bit high products.
// The result's larger component lies in [2^56, 2^61], so a 32-bit leading-
// zero count of the high words renormalises it.
__device__ __forceinline__ void ix_mul(long long& X, long long& Y, int& e, long long a, long long b, int f) {
  const int xh = (int)(X >> 32), yh = (int)(Y >> 32), ah = (int)(a >> 32), bh = (int)(b >> 32);
  const int xl = (int)((unsigned)X >> 2), yl = (int)((unsigned)Y >> 2);
  const int al = (int)((unsigned)a >> 2), bl = (int)((unsigned)b >> 2);
  long long re = (long long)xh * ah - (long long)yh * bh;
  long long im = (long long)xh * bh + (long long)yh * ah;
  const long long mr = (long long)xh * al + (long long)xl * ah - (long long)yh * bl - (long long)yl * bh;
  const long long mi = (long long)xh * bl + (long long)xl * bh + (long long)yh * al + (long long)yl * ah;
  re += mr >> 30;
  im += mi >> 30;
  const int rh = (int)(re >> 32), ih = (int)(im >> 32);
  const unsigned m = (unsigned)(rh ^ (rh >> 31)) | (unsigned)(ih ^ (ih >> 31));
  const int kz = __clz((int)m) - 2;  // 0..8 for a non-zero product; 30 for zero
  X = ix_shl(re, kz);
  Y = ix_shl(im, kz);
  e += f + 64 - kz;
}

// (X + iY) 2^e = prod_{i < K} (vr_i + i vi_i) (e relative to the rows' scales),
// in interleaved blocks joined at the end, so that independent dependency
// chains are in flight: three for long blocks (K >= 24; measured 3 % faster
// at n = 40), two for shorter ones (3 % faster at the batch study's orders).
template <int N, int K>
__device__ __forceinline__ void ix_product(const long long (&vr)[N], const long long (&vi)[N], long long& X,
                                           long long& Y, int& e) {
  constexpr int C = K >= 24 ? 3 : 2;
  const int k0 = ix_shift(vr[0], vi[0]);
  X = ix_shl(vr[0], k0);
  Y = ix_shl(vi[0], k0);
  e = -k0;
  if constexpr (K == 1) return;
  const int k1 = ix_shift(vr[1], vi[1]);
  long long U = ix_shl(vr[1], k1), V = ix_shl(vi[1], k1);
  int g = -k1;
  if constexpr (C == 2) {
#pragma unroll
    for (int i = 2; i < K; ++i) {
      const int kf = ix_shift(vr[i], vi[i]);
      const long long a = ix_shl(vr[i], kf), b = ix_shl(vi[i], kf);
      if (i & 1)
        ix_mul(U, V, g, a, b, -kf);
      else
        ix_mul(X, Y, e, a, b, -kf);
    }
  } else {
    const int k2 = ix_shift(vr[2], vi[2]);
    long long P = ix_shl(vr[2], k2), Q = ix_shl(vi[2], k2);
    int h = -k2;
#pragma unroll
    for (int i = 3; i < K; ++i) {
      const int kf = ix_shift(vr[i], vi[i]);
      const long long a = ix_shl(vr[i], kf), b = ix_shl(vi[i], kf);
      if (i % 3 == 0)
        ix_mul(X, Y, e, a, b, -kf);
      else if (i % 3 == 1)
        ix_mul(U, V, g, a, b, -kf);
      else
        ix_mul(P, Q, h, a, b, -kf);
    }
    ix_mul(U, V, g, P, Q, h);
  }
  ix_mul(X, Y, e, U, V, g);
}

// Exponent offset of the integer block: sum over its rows of (eb_i - 1086).
template <int N>
__device__ __forceinline__ int ix_offset(const int* sEb) {
  int c = 0;
#pragma unroll 1
  for (int i = 0; i < kIxRows<N>; ++i) c += sEb[i] - 1086;
  return c;
}

// Product of w_i = v_i 2^(eb_i - 1086): the first kIxRows<N> factors from the
// integer block, the others in FP64 (two interleaved chains; RN selects how
// their doubles are rounded).
template <int N, bool RN>
struct FxProduct<N, true, kProdF64, RN> {
  static constexpr int K = kIxRows<N>;

  static __device__ __forceinline__ void eval(const long long (&vr)[N], const long long (&vi)[N], const int* sEb,
                                              double& pr, double& pi, double z) {
    eval(vr, vi, sEb, pr, pi, z, K > 0 ? ix_offset<N>(sEb) : 0);
  }

  // ixc: ix_offset<N>(sEb), computed once by the caller
  static __device__ __forceinline__ void eval(const long long (&vr)[N], const long long (&vi)[N], const int* sEb,
                                              double& pr, double& pi, double z, int ixc) {
    if constexpr (K == 0) {
      double ar = fx_to_double<RN>(vr[0], sEb[0]), ai = fx_to_double<RN>(vi[0], sEb[0]);
      if constexpr (N == 1) {
        pr = ar;
        pi = ai;
      } else {
        double br = fx_to_double<RN>(vr[1], sEb[1]), bi = fx_to_double<RN>(vi[1], sEb[1]);
#pragma unroll
        for (int i = 2; i < N; ++i) {
          const int eb = sEb[i];
          const double cr = fx_to_double<RN>(vr[i], eb), ci = fx_to_double<RN>(vi[i], eb);
          if (i & 1)
            cmul(br, bi, cr, ci, z);
          else
            cmul(ar, ai, cr, ci, z);
        }
        cmul(ar, ai, br, bi, z);
        pr = ar;
        pi = ai;
      }
    } else if constexpr (K == N) {
      long long X, Y;
      int e;
      ix_product<N, K>(vr, vi, X, Y, e);
      const int et = e + ixc;
      pr = scalbn((double)X, et);
      pi = scalbn((double)Y, et);
    } else {
      static_assert(N - K >= 2, "the FP64 part keeps two chains");
      long long X, Y;
      int e;
      ix_product<N, K>(vr, vi, X, Y, e);
      double ar = fx_to_double<RN>(vr[K], sEb[K]), ai = fx_to_double<RN>(vi[K], sEb[K]);
      double br = fx_to_double<RN>(vr[K + 1], sEb[K + 1]), bi = fx_to_double<RN>(vi[K + 1], sEb[K + 1]);
#pragma unroll
      for (int i = K + 2; i < N; ++i) {
        const int eb = sEb[i];
        const double cr = fx_to_double<RN>(vr[i], eb), ci = fx_to_double<RN>(vi[i], eb);
        if ((i - K) & 1)
          cmul(br, bi, cr, ci, z);
        else
          cmul(ar, ai, cr, ci, z);
      }
      cmul(ar, ai, br, bi, z);
      const int et = e + ixc;
      cmul(ar, ai, scalbn((double)X, et), scalbn((double)Y, et), z);
      pr = ar;
      pi = ai;
    }
  }
};

template <int N, bool RN>
struct FxProduct<N, false, kProdF64, RN> {
  static __device__ __forceinline__ void eval(const long long (&v)[N], const int* sEb, double& p, double z) {
    double a = fx_to_double<RN>(v[0], sEb[0]);
    if constexpr (N == 1) {
      p = a;
    } else {
      double b = fx_to_double<RN>(v[1], sEb[1]);
#pragma unroll
      for (int i = 2; i < N; ++i) {
        const double c = fx_to_double<RN>(v[i], sEb[i]);
        if (i & 1)
          b = fma(b, c, z);
        else
          a = fma(a, c, z);
      }
      p = fma(a, b, z);
    }
  }
};

// FP32 significands straight from the integers; exponents add in integers.
template <int N, bool RN>
struct FxProduct<N, true, kProdF32, RN> {
  static __device__ __forceinline__ void eval(const long long (&vr)[N], const long long (&vi)[N], const int* sEb,
                                              double& pr, double& pi, double z, int) {
    eval(vr, vi, sEb, pr, pi, z);
  }
  static __device__ __forceinline__ void eval(const long long (&vr)[N], const long long (&vi)[N], const int* sEb,
                                              double& pr, double& pi, double) {
    float ar = 1.f, ai = 0.f, br = 1.f, bi = 0.f;
    int E = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const unsigned long long sr = (unsigned long long)(vr[i] >> 63), si = (unsigned long long)(vi[i] >> 63);
      const int lzr = __clzll((long long)((vr[i] ^ sr) - sr));
      const int lzi = __clzll((long long)((vi[i] ^ si) - si));
      const int lzref = min(lzr, lzi);
      const float fr = fx_to_f32(vr[i], lzref);
      const float fi = fx_to_f32(vi[i], lzref);
      // |w_i| = |f| 2^(63 - lzref + eb_i - 1086)
      E += 63 - lzref + sEb[i] - 1086;
      if (i == 0) {
        ar = fr, ai = fi;
      } else if (i == 1) {
        br = fr, bi = fi;
      } else if (i & 1) {
        cmulf(br, bi, fr, fi);
      } else {
        cmulf(ar, ai, fr, fi);
      }
    }
    if constexpr (N > 1) cmulf(ar, ai, br, bi);
    pr = f32_times_pow2(ar, E);
    pi = f32_times_pow2(ai, E);
  }
};

template <int N, bool RN>
struct FxProduct<N, false, kProdF32, RN> {
  static __device__ __forceinline__ void eval(const long long (&v)[N], const int* sEb, double& p, double) {
    float a = 1.f, b = 1.f;
    int E = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const unsigned long long s = (unsigned long long)(v[i] >> 63);
      const int lz = __clzll((long long)((v[i] ^ s) - s));
      const float f = fx_to_f32(v[i], lz);
      E += 63 - lz + sEb[i] - 1086;
      if (i & 1)
        b *= f;
      else
        a *= f;
    }
    p = f32_times_pow2(a * b, E);
  }
};

// Stage: per-row scale exponents, the +-2A tables and v0, from global memory.
// Returns (block-uniform) whether any entry is non-finite.
template <int N, bool CPLX>
__device__ __forceinline__ bool fx_stage(const double* __restrict__ A, long long* sP, long long* sM, long long* sV0,
                                         int* sEb, int* sF, int* status) {
  constexpr int E = CPLX ? 2 : 1;
  constexpr int S = FxShape<N, CPLX>::S;
  int bad = 0;
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
    double mx = 0.0;
#pragma unroll
    for (int c = 0; c < E; ++c) {
      double s = 0.0;
      for (int j = 0; j < N; ++j) {
        const double v = A[((size_t)i * N + j) * E + c];
        bad |= not_finite(v) ? 1 : 0;
        s += fabs(v);
      }
      mx = fmax(mx, s);
    }
    // 2^F_i with sum_j |a_ij| 2^F_i < 2^62: F_i = 61 - floor(log2 max_c sum_j |a_ij|)
    int F = 0;
    if (mx > 0.0 && !bad) {
      const int ex = dexp_of(mx);
      F = ex == 0 ? 61 + 1022 : 61 - (ex - 1023);  // subnormal sums: scale as the smallest normal
    }
    sF[i] = F;
    sEb[i] = 1086 - F - 1;  // the extra -1 halves v = 2w into w
  }
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) atomicOr(status, (int)kStatusNonFinite);
    return true;
  }
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const int F = sF[i];
#pragma unroll
    for (int c = 0; c < E; ++c) {
      const long long q = __double2ll_rn(scalbn(A[(size_t)idx * E + c], F));
      sP[(j * S + i) * E + c] = 2 * q;
      sM[(j * S + i) * E + c] = -2 * q;
    }
  }
  __syncthreads();
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
#pragma unroll
    for (int c = 0; c < E; ++c) {
      // v0_i = A_{i,n} - sum_{j<n} A_ij  (all e_j = -1), from the doubled table
      long long s = sP[((N - 1) * S + i) * E + c];
      for (int j = 0; j < N - 1; ++j) s -= sP[(j * S + i) * E + c];
      sV0[i * E + c] = s / 2;
    }
  }
  __syncthreads();
  return false;
}

// TWO_TABLES: read -2A from its own table; otherwise negate +2A on the fly
// (integer ops only; used where shared memory is tight).  ST: column stride
// of the tables in entries.
template <int N, int MODE, bool TWO_TABLES = true, int ST = N>
__device__ __forceinline__ void thread_walk_c128_fx(const longlong2* __restrict__ sP, const longlong2* __restrict__ sM,
                                                    const longlong2* __restrict__ sV0, const int* __restrict__ sEb,
                                                    uint64_t r, const uint64_t end, dd& accr, dd& acci) {
  if (r >= end) return;
  const double z = fx_to_double(sV0[0].x, sEb[0]) * 0.0;  // a register zero (+-0.0) for the product FMAs
  const int ixc = MODE == kProdF64 ? ix_offset<N>(sEb) : 0;
  long long vr[N], vi[N];
  {
    // seed once (App. A steps 2, 5-8, in v = 2w form): exact, never redone
    const uint64_t x = r ^ (r >> 1);
    longlong2 seed[N];
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      longlong2 v = sV0[i];
#pragma unroll 1
      for (int j = 0; j < N - 1; ++j) {
        if ((x >> j) & 1ull) {
          const longlong2 c = sP[j * ST + i];
          v.x += c.x;
          v.y += c.y;
        }
      }
      seed[i] = v;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      vr[i] = seed[i].x;
      vi[i] = seed[i].y;
    }
  }
  while (r < end) {
    const uint64_t run_end = min(end, (r | (kRun - 1)) + 1);
    double sr = 0.0, si = 0.0;
    uint32_t odd = (uint32_t)(r & 1ull);
    for (; r < run_end; ++r) {
      double pr, pi;
      FxProduct<N, true, MODE>::eval(vr, vi, sEb, pr, pi, z, ixc);
      const double sg = pm_one(odd);
      odd ^= 1u;
      sr = fma(sg, pr, sr);
      si = fma(sg, pi, si);
      int j;
      uint32_t neg;
      gray_step(r, j, neg);
      if constexpr (TWO_TABLES) {
        const longlong2* col = (neg ? sM : sP) + j * ST;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const longlong2 c = col[i];
          vr[i] += c.x;
          vi[i] += c.y;
        }
      } else {
        const longlong2* col = sP + j * ST;
        const long long m = -(long long)neg;  // 0 or all ones
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const longlong2 c = col[i];
          vr[i] += (c.x ^ m) - m;
          vi[i] += (c.y ^ m) - m;
        }
      }
    }
    accr = dd_add_d(accr, sr);
    acci = dd_add_d(acci, si);
  }
}

// Warp-level staging of one complex matrix of order n (<= 32) into a warp's
// own slot: row scales, the +2A table (column-major) and v0.  Returns whether
// any entry is non-finite (warp-uniform).
__device__ __forceinline__ bool fx_stage_warp_c128(const double2* __restrict__ A, int n, longlong2* sP, longlong2* sV0,
                                                   int* sEb, int* sF) {
  const int lane = threadIdx.x & 31;
  int bad = 0;
  if (lane < n) {
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < n; ++j) {
      const double2 v = A[lane * n + j];
      bad |= (not_finite(v.x) || not_finite(v.y)) ? 1 : 0;
      sr += fabs(v.x);
      si += fabs(v.y);
    }
    const double mx = fmax(sr, si);
    int F = 0;
    if (mx > 0.0 && !bad) {
      const int ex = dexp_of(mx);
      F = ex == 0 ? 61 + 1022 : 61 - (ex - 1023);
    }
    sF[lane] = F;
    sEb[lane] = 1086 - F - 1;
  }
  if (__any_sync(0xffffffffu, bad)) return true;
  __syncwarp();
  for (int idx = lane; idx < n * n; idx += 32) {
    const int i = idx / n, j = idx - i * n;
    const int F = sF[i];
    const double2 v = A[idx];
    sP[j * n + i] = make_longlong2(2 * __double2ll_rn(scalbn(v.x, F)), 2 * __double2ll_rn(scalbn(v.y, F)));
  }
  __syncwarp();
  if (lane < n) {
    longlong2 s = sP[(n - 1) * n + lane];
    for (int j = 0; j < n - 1; ++j) {
      s.x -= sP[j * n + lane].x;
      s.y -= sP[j * n + lane].y;
    }
    sV0[lane] = make_longlong2(s.x / 2, s.y / 2);
  }
  __syncwarp();
  return false;
}

template <int N, int MODE, int ST = N>
__device__ __forceinline__ void thread_walk_r64_fx(const long long* __restrict__ sP, const long long* __restrict__ sM,
                                                   const long long* __restrict__ sV0, const int* __restrict__ sEb,
                                                   uint64_t r, const uint64_t end, dd& accr) {
  if (r >= end) return;
  const double z = fx_to_double(sV0[0], sEb[0]) * 0.0;
  long long v[N];
  {
    const uint64_t x = r ^ (r >> 1);
    long long seed[N];
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      long long s = sV0[i];
#pragma unroll 1
      for (int j = 0; j < N - 1; ++j)
        if ((x >> j) & 1ull) s += sP[j * ST + i];
      seed[i] = s;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = seed[i];
  }
  while (r < end) {
    const uint64_t run_end = min(end, (r | (kRun - 1)) + 1);
    double s = 0.0;
    uint32_t odd = (uint32_t)(r & 1ull);
    for (; r < run_end; ++r) {
      double p;
      FxProduct<N, false, MODE>::eval(v, sEb, p, z);
      s = fma(pm_one(odd), p, s);
      odd ^= 1u;
      int j;
      uint32_t neg;
      gray_step(r, j, neg);
      const long long* col = (neg ? sM : sP) + j * ST;
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] += col[i];
    }
    accr = dd_add_d(accr, s);
  }
}

template <int N, bool CPLX, int MODE>
__global__ void __launch_bounds__(kWalkThreads) k_walk_fx(const double* __restrict__ A, uint64_t first, uint64_t count,
                                                          double* __restrict__ partials, int accumulate,
                                                          int* __restrict__ status) {
  constexpr int E = CPLX ? 2 : 1;
  constexpr int S = FxShape<N, CPLX>::S;
  using Shape = FxShape<N, CPLX>;
  extern __shared__ __align__(16) long long fsm[];
  char* base = reinterpret_cast<char*>(fsm);
  long long* sP = fsm;
  long long* sM = sP + N * S * E;
  long long* sV0 = reinterpret_cast<long long*>(base + Shape::v0_off);
  int* sEb = reinterpret_cast<int*>(base + Shape::eb_off);
  int* sF = reinterpret_cast<int*>(base + Shape::f_off);
  dd* sRed = reinterpret_cast<dd*>(fsm);  // reused after the walk (tables no longer read)

  const bool bad = fx_stage<N, CPLX>(A, sP, sM, sV0, sEb, sF, status);

  // FP64 products multiply the unscaled row values v_i 2^-63 (below 1/2 in
  // magnitude, so no chain leaves the double range however the rows are
  // scaled); the rows' scales 2^(eb_i - 1023) are applied once, to the
  // thread's sum.  The FP32-product mode carries its exponents in integers.
  const int* sE = sEb;
  int scale = 0;
  if constexpr (MODE == kProdF64) {
    if (!bad) {
      for (int i = 0; i < N; ++i) scale += sEb[i] - 1023;
      if (threadIdx.x < N) sF[threadIdx.x] = 1023;  // sF is free after staging
      __syncthreads();
      sE = sF;
    }
  }

  uint64_t r, end;
  thread_range(first, count, r, end);
  dd accr{0.0, 0.0}, acci{0.0, 0.0};
  if (!bad) {
    if constexpr (CPLX)
      thread_walk_c128_fx<N, MODE, true, S>(reinterpret_cast<const longlong2*>(sP),
                                            reinterpret_cast<const longlong2*>(sM),
                                            reinterpret_cast<const longlong2*>(sV0), sE, r, end, accr, acci);
    else
      thread_walk_r64_fx<N, MODE, S>(sP, sM, sV0, sE, r, end, accr);
    if constexpr (MODE == kProdF64) {
      accr = dd{scalbn(accr.hi, scale), scalbn(accr.lo, scale)};
      acci = dd{scalbn(acci.hi, scale), scalbn(acci.lo, scale)};
    }
  } else {
    accr = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
    acci = accr;
  }
  __syncthreads();  // every thread is done with the tables before they are reused
  block_store<CPLX>(accr, acci, sRed, partials, accumulate);
}

template <int N, bool CPLX, int MODE>
struct FxKernel {
  static constexpr size_t smem = FxShape<N, CPLX>::smem_bytes;

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
      e = cudaFuncSetAttribute(k_walk_fx<N, CPLX, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_fx<N, CPLX, MODE>, kWalkThreads, smem);
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
    k_walk_fx<N, CPLX, MODE><<<a.blocks, kWalkThreads, smem, a.stream>>>(a.A, a.first, a.count, a.partials,
                                                                         a.accumulate, a.status);
    return cudaGetLastError();
  }
};

template <bool CPLX, int MODE, int LO, int HI>
cudaError_t fx_dispatch(const WalkArgs& a) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    if (a.n == LO) return FxKernel<LO, CPLX, MODE>::launch(a);
    return fx_dispatch<CPLX, MODE, LO + 1, HI>(a);
  }
}

template <bool CPLX, int MODE, int LO, int HI>
int fx_blocks_dispatch(int n) {
  if constexpr (LO > HI) {
    return 0;
  } else {
    if (n == LO) return FxKernel<LO, CPLX, MODE>::resident_blocks();
    return fx_blocks_dispatch<CPLX, MODE, LO + 1, HI>(n);
  }
}

}  // namespace perm

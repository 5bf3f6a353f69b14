// Gray-code walks with packed double-float products (the same sum as
// glynn_walk.cuh: Sec. 2.A, App. A), in two row-sum arithmetics.
//
// Packing.  Rows 2k and 2k+1 share one 64-bit register pair per component
// (the .x and .y lanes of a float2), so each packed FP32 instruction of
// sm_100+ (add/sub/mul/fma .f32x2) works on two rows.  On GB300 a packed FMA
// issues at half the scalar rate but does two FMAs, so the FP32 pipe does the
// same work with half the instructions.  The product Prod_i v_i runs as six
// double-float chains held in three packed chain pairs: chain pair c
// multiplies the row pairs c, c+3, c+6, ... (each step a complex double-float
// product: exact FP32 products by FMA, TwoSum for the sums, about 48
// significant bits); the chains are renormalised by powers of two every eight
// factors and at the end, multiplied together, and the term is rebuilt as
// FP64 (high and low parts converted and scaled by 2^E with the sign folded
// in) and summed into FP64 run sums folded into double-double.
//
// Row scale.  Row i of A is scaled by 2^G_i so that max(sum_j |Re a_ij|,
// sum_j |Im a_ij|) 2^G_i < 1; every row sum in Glynn's form v_i = sum_j e_j
// a_ij (e_n = +1) then lies in the unit square.
//
// Double-float rows (the default of the two, kRowsPdf).  Each row sum is an
// unevaluated pair of floats renormalised after every step (TwoSum, then
// FastTwoSum: about 48 significant bits relative to the row sum itself), the
// columns are the double-float roundings of the exact integer columns, and
// every 1024 codes (pdf_tile_log()) each row is re-seeded from its exact
// int64 value (entries rounded once to 2^-61 of the row scale, as fine as the
// fixed-point walk), so the rounding errors of the steps stay independent and
// average out over the sum.
//
// Exact float-pair rows (kRowsPair).  Each scaled entry is rounded once to
// the grid 2^-47 (a 48-bit fixed point relative to the row's largest possible
// sum), so every row sum is an exact multiple of 2^-47 held as h + l with h
// on the grid 2^-23 (at most 24 significant bits) and l on the grid 2^-47
// with |l| <= 2^-24.  A Gray step adds a column c = ch + cl split the same
// way: h + ch and l + cl are exact float additions, and a carry (l rounded to
// the grid 2^-23 with the 1.5 magic constant) moves from l to h exactly.
// These rows never drift and are seeded once per thread, at six packed
// operations per step instead of eleven; but the 48-bit rounding of the
// entries is a fixed perturbation of the matrix, which does not average out
// (about 1e-11 relative at n = 40 instead of 1e-13).
//
// Warp-uniform steps.  Thread ranges are congruent modulo 2^8 codes, so the
// lanes of a warp flip the same column with the same sign on all but one step
// in 128: the column read is a shared-memory broadcast.
//
// The number of packed chain pairs (3) was measured against 2 and 4 at
// n = 40 and 48: 3 is 3 % faster than 2 at n = 40 and equal at 48; 4 spills
// at n = 48.  Renormalising the rows every second step instead of every step
// (saving 3 of the 11 packed operations of half the updates) measured 3 %
// slower, with the step loop unrolled by two.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include <cstdint>

#include "dd.cuh"
#include "glynn_walk.cuh"
#include "glynn_walk_df.cuh"
#include "perm_internal.h"

namespace perm {

constexpr int kXpGrid = 47;       // exact float-pair rows: multiples of 2^-47 of the row scale
constexpr int kPdfGrid = 61;      // double-float rows: exact int64 seeds in units of 2^-61 of the row scale
// double-float rows: re-seeded every 2^tile_log codes (a kernel argument: pdf_tile_log())
constexpr int kXpAlignLog = 8;    // thread ranges are congruent modulo 2^8 codes
constexpr int kXpRenormEvery = 8; // chain renormalisation period (factors)
#ifndef PERM_XP_CHAIN_PAIRS
#define PERM_XP_CHAIN_PAIRS 3
#endif

constexpr int kXpChainPairs = PERM_XP_CHAIN_PAIRS;  // packed chain pairs of the product

template <int N>
constexpr int kPairs = (N + 1) / 2;  // row pairs (an odd order gets a constant row 1)

template <int N, bool EXACT>
struct XpShape {
  static constexpr int NP = kPairs<N>;
  // +c and -c tables: [column j < N][pair k][re, im] float4 (h.x, h.y, l.x, l.y)
  static constexpr size_t table_f4 = (size_t)N * NP * 2;
  // exact rows: the seed pairs [k][re, im] float4; double-float rows: the
  // int64 columns [j][k][lane] longlong2 (re, im) and seeds [k][lane]
  static constexpr size_t seed_bytes =
      EXACT ? (size_t)NP * 2 * sizeof(float4) : ((size_t)N * NP * 2 + (size_t)NP * 2) * sizeof(longlong2);
  static constexpr size_t smem_bytes = 2 * table_f4 * sizeof(float4) + seed_bytes + 8 * sizeof(dd) + 16;
};

// ---- packed FP32 helpers (sm_100+: two FP32 operations per instruction) ----
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Two complex double-float numbers side by side (lanes .x and .y).
struct P4 {
  float2 hr, lr, hi, li;
};

// Exact add of a column pair to a row pair on the fixed grids (see header).
__device__ __forceinline__ void xp_add(float2& h, float2& l, float2 ch, float2 cl) {
  const float2 magic = make_float2(1.5f, 1.5f);  // ulp 2^-23: rounds to the grid of h
  h = f2add(h, ch);
  l = f2add(l, cl);
  const float2 c = f2sub(f2add(l, magic), magic);
  h = f2add(h, c);
  l = f2sub(l, c);
}

__device__ __forceinline__ void xp_add_col(P4& v, const float4& re, const float4& im) {
  xp_add(v.hr, v.lr, make_float2(re.x, re.y), make_float2(re.z, re.w));
  xp_add(v.hi, v.li, make_float2(im.x, im.y), make_float2(im.z, im.w));
}

// Double-float add of a column pair to a row pair: TwoSum of the high parts,
// the low parts added to its error, then FastTwoSum renormalisation.
__device__ __forceinline__ void df2_add(float2& h, float2& l, float2 ch, float2 cl) {
  const float2 s = f2add(h, ch);
  const float2 bb = f2sub(s, h);
  float2 e = f2add(f2sub(h, f2sub(s, bb)), f2sub(ch, bb));
  e = f2add(e, f2add(l, cl));
  h = f2add(s, e);
  l = f2sub(e, f2sub(h, s));
}

__device__ __forceinline__ void df2_add_col(P4& v, const float4& re, const float4& im) {
  df2_add(v.hr, v.lr, make_float2(re.x, re.y), make_float2(re.z, re.w));
  df2_add(v.hi, v.li, make_float2(im.x, im.y), make_float2(im.z, im.w));
}

// a * b for two packed complex double-floats: exact products by FMA, TwoSum for
// the real and imaginary sums; the low parts are left unrenormalised (within a
// few units of the last place of the high parts), as the next product takes them.
__device__ __forceinline__ P4 p4_mul(const P4& a, const P4& b) {
  P4 r;
  {
    const float2 p1 = f2mul(a.hr, b.hr);
    float2 e1 = f2fma(a.hr, b.hr, f2neg(p1));
    e1 = f2fma(a.hr, b.lr, e1);
    e1 = f2fma(a.lr, b.hr, e1);
    const float2 p2 = f2mul(a.hi, b.hi);
    float2 e2 = f2fma(a.hi, b.hi, f2neg(p2));
    e2 = f2fma(a.hi, b.li, e2);
    e2 = f2fma(a.li, b.hi, e2);
    // TwoSum(p1, -p2)
    const float2 s = f2sub(p1, p2);
    const float2 bb = f2sub(s, p1);
    const float2 err = f2sub(f2sub(p1, f2sub(s, bb)), f2add(p2, bb));
    r.hr = s;
    r.lr = f2add(err, f2sub(e1, e2));
  }
  {
    const float2 p3 = f2mul(a.hr, b.hi);
    float2 e3 = f2fma(a.hr, b.hi, f2neg(p3));
    e3 = f2fma(a.hr, b.li, e3);
    e3 = f2fma(a.lr, b.hi, e3);
    const float2 p4 = f2mul(a.hi, b.hr);
    float2 e4 = f2fma(a.hi, b.hr, f2neg(p4));
    e4 = f2fma(a.hi, b.lr, e4);
    e4 = f2fma(a.li, b.hr, e4);
    // TwoSum(p3, p4)
    const float2 s = f2add(p3, p4);
    const float2 bb = f2sub(s, p3);
    const float2 err = f2add(f2sub(p3, f2sub(s, bb)), f2sub(p4, bb));
    r.hi = s;
    r.li = f2add(err, f2add(e3, e4));
  }
  return r;
}

// Scale each lane's complex value by a power of two so that the larger of its
// high parts lies in [1, 2); the exponents removed are added to ex, ey.  A
// lane whose high parts are zero (or subnormal) is left as it is.
__device__ __forceinline__ void p4_renorm(P4& a, int& ex, int& ey) {
  const int rx = (__float_as_int(a.hr.x) >> 23) & 0xff, ix = (__float_as_int(a.hi.x) >> 23) & 0xff;
  const int ry = (__float_as_int(a.hr.y) >> 23) & 0xff, iy = (__float_as_int(a.hi.y) >> 23) & 0xff;
  int mx = max(rx, ix), my = max(ry, iy);
  mx = mx ? mx : 127;
  my = my ? my : 127;
  const float2 sc = make_float2(__int_as_float((254 - mx) << 23), __int_as_float((254 - my) << 23));
  a.hr = f2mul(a.hr, sc);
  a.lr = f2mul(a.lr, sc);
  a.hi = f2mul(a.hi, sc);
  a.li = f2mul(a.li, sc);
  ex += mx - 127;
  ey += my - 127;
}

// +-2^E as a double from integer bits (E within the normal range).
__device__ __forceinline__ double signed_pow2(int E, uint32_t negative) {
  return __hiloint2double((int)(((uint32_t)(1023 + E) << 20) | (negative << 31)), 0);
}

// (-1)^negative f 2^E as a double, built from the bits of the float f with
// integer instructions only (the FP64 pipe, at 1/64 of the FP32 rate here,
// would convert it): sign flipped, exponent field re-biased from 127 to 1023
// plus E, the 23 fraction bits moved to the top of the 52.  Exact.  Zero and
// subnormal floats, and results below the normal double range, give zero (a
// term part below 2^-1022 of the permanent's scale).  E must not take the
// result above the double range.
__device__ __forceinline__ double f32_scaled_f64(float f, int E, uint32_t negative) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t mag = u & 0x7FFFFFFFu;
  const int be = (int)(mag >> 23) + 896 + E;  // biased double exponent
  const uint32_t hi = ((u ^ (negative << 31)) & 0x80000000u) | ((mag >> 3) + ((uint32_t)(896 + E) << 20));
  const bool zero = mag < 0x00800000u || be <= 0;
  return __hiloint2double(zero ? 0 : (int)hi, zero ? 0 : (int)(u << 29));
}

// Product of the N row sums (NP packed pairs) as FP64 parts scaled by
// 2^E: on return p = (pr_hi + pr_lo) + i (pi_hi + pi_lo) times 2^E.
template <int N>
__device__ __forceinline__ void xp_product(const P4 (&v)[kPairs<N>], cdf& z, int& E) {
  constexpr int NP = kPairs<N>;
  constexpr int CP = NP >= kXpChainPairs ? kXpChainPairs : NP;  // packed chain pairs
  P4 c[CP];
  int ex[CP], ey[CP];
  int len[CP];
#pragma unroll
  for (int q = 0; q < CP; ++q) c[q] = v[q], ex[q] = 0, ey[q] = 0, len[q] = 1;
#pragma unroll
  for (int k = CP; k < NP; ++k) {
    const int q = k % CP;
    c[q] = p4_mul(c[q], v[k]);
    if (++len[q] % kXpRenormEvery == 0 && k + CP < NP) p4_renorm(c[q], ex[q], ey[q]);
  }
#pragma unroll
  for (int q = 0; q < CP; ++q) p4_renorm(c[q], ex[q], ey[q]);
#pragma unroll
  for (int q = 1; q < CP; ++q) {
    c[0] = p4_mul(c[0], c[q]);
    ex[0] += ex[q];
    ey[0] += ey[q];
  }
  const cdf x{c[0].hr.x, c[0].lr.x, c[0].hi.x, c[0].li.x};
  const cdf y{c[0].hr.y, c[0].lr.y, c[0].hi.y, c[0].li.y};
  z = cdf_mul(x, y);
  E = ex[0] + ey[0];
}

// Row scales 2^G_i (sG) of the staging step (E = 2: complex entries, 1:
// real).  Returns (block-uniform) whether any entry is non-finite.
template <int N, int E = 2>
__device__ __forceinline__ bool xp_row_scales(const double* __restrict__ A, int* sG, int* status) {
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
    // 2^G_i with mx 2^G_i in (1/2, 1]: G_i = -(floor(log2 mx) + 1), exact powers of two kept
    int G = 0;
    if (mx > 0.0 && !bad) {
      int e;
      const double f = frexp(mx, &e);  // mx = f 2^e, f in [1/2, 1)
      G = -e;
      (void)f;
    }
    sG[i] = G;
  }
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) atomicOr(status, (int)kStatusNonFinite);
    return true;
  }
  return false;
}

// Stage for exact float-pair rows: the +c / -c tables on the 2^-47 grid and
// the seed pairs.  Returns whether any entry is non-finite.
template <int N>
__device__ __forceinline__ bool xp_stage_exact(const double* __restrict__ A, float4* sP, float4* sM, float4* sV0,
                                               int* sG, int* status) {
  constexpr int NP = kPairs<N>;
  if (xp_row_scales<N>(A, sG, status)) return true;
  float* fP = reinterpret_cast<float*>(sP);
  float* fM = reinterpret_cast<float*>(sM);
  // Column entries c_ij = 2 a_ij 2^G_i on the 2^-47 grid, as float pairs.
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const int G = sG[i];
    const int k = i >> 1, lane = i & 1;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float h = 0.f, l = 0.f;
      if (j < N - 1) {
        const long long q = __double2ll_rn(scalbn(A[(size_t)idx * 2 + c], G + kXpGrid));
        const long long C = 2 * q;                              // |C| <= 2^48
        const long long kh = (C + (1ll << 23)) >> 24;            // nearest multiple of 2^24
        const long long m = C - (kh << 24);                      // |m| <= 2^23
        h = (float)kh * 0x1p-23f;                                 // exact: |kh| <= 2^24
        l = (float)m * 0x1p-47f;                                  // exact: |m| <= 2^23
      }
      const size_t base = (((size_t)j * NP + k) * 2 + c) * 4;
      fP[base + lane] = h;
      fP[base + 2 + lane] = l;
      fM[base + lane] = -h;
      fM[base + 2 + lane] = -l;
    }
  }
  // The missing row of an odd order: constant 1 (h = 1, l = 0; columns zero).
  if (N & 1) {
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const size_t base = (((size_t)j * NP + (NP - 1)) * 2 + c) * 4;
        fP[base + 1] = 0.f, fP[base + 3] = 0.f;
        fM[base + 1] = 0.f, fM[base + 3] = 0.f;
      }
    }
  }
  // Seed pairs: v0_i = a_{i,n} - sum_{j<n} a_ij on the grid (all e_j = -1).
  float* fV = reinterpret_cast<float*>(sV0);
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
    const int G = sG[i];
    const int k = i >> 1, lane = i & 1;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      long long s = 0;
      for (int j = 0; j < N; ++j) {
        const long long q = __double2ll_rn(scalbn(A[((size_t)i * N + j) * 2 + c], G + kXpGrid));
        s += (j == N - 1) ? q : -q;
      }
      const long long kh = (s + (1ll << 23)) >> 24;
      const long long m = s - (kh << 24);
      fV[(k * 2 + c) * 4 + lane] = (float)kh * 0x1p-23f;
      fV[(k * 2 + c) * 4 + 2 + lane] = (float)m * 0x1p-47f;
    }
  }
  if ((N & 1) && threadIdx.x == 0) {
    // constant row 1 + 0i in the odd lane of the last pair
    fV[((NP - 1) * 2 + 0) * 4 + 1] = 1.0f;
    fV[((NP - 1) * 2 + 0) * 4 + 3] = 0.0f;
    fV[((NP - 1) * 2 + 1) * 4 + 1] = 0.0f;
    fV[((NP - 1) * 2 + 1) * 4 + 3] = 0.0f;
  }
  __syncthreads();
  return false;
}

// Double-float pair (h, l) of v 2^-61 for an int64 v with |v| <= 2^62, with
// integer and FP32 instructions only (the FP64 pipe runs at 1/64 of the FP32
// rate on this part, and a re-seed converts every row).  v = a 2^46 + b 2^23 + c
// with a = v >> 46 (signed, |a| <= 2^16) and b, c unsigned 23-bit fields.  Each
// part is an exact float: a field placed in the significand of a power of two
// P = 2^(23+k) (or added to 1.5 P, for the signed a) reads P + field 2^k
// exactly, and subtracting P leaves field 2^k.  The parts do not overlap and
// |a 2^-15| >= 2^-15 > b 2^-38 > c 2^-61 whenever the larger part is non-zero,
// so two FastTwoSums (Dekker) sum them into a normalised pair; only the low
// word's own addition rounds (about 2^-48 relative to v).
__device__ __forceinline__ void pdf_split(long long v, float& h, float& l) {
  const int a = (int)(v >> 46);
  const unsigned b = (unsigned)((unsigned long long)v >> 23) & 0x7FFFFFu;
  const unsigned c = (unsigned)v & 0x7FFFFFu;
  const float fa = __fsub_rn(__int_as_float(0x43C00000 + a), 384.0f);               // 1.5 2^8, ulp 2^-15
  const float fb = __fsub_rn(__int_as_float(0x38000000 | (int)b), 0x1p-15f);         // 2^-15, ulp 2^-38
  const float fc = __fsub_rn(__int_as_float(0x2C800000 | (int)c), 0x1p-38f);         // 2^-38, ulp 2^-61
  const float s = __fadd_rn(fa, fb);
  const float e = __fsub_rn(fb, __fsub_rn(s, fa));
  const float t = __fadd_rn(e, fc);
  h = __fadd_rn(s, t);
  l = __fsub_rn(t, __fsub_rn(h, s));
}

// Stage for double-float rows: Q_ij = rint(a_ij 2^(G_i + 61)) (|Q| <= 2^61),
// the int64 columns 2 Q_ij (sQ, [k][j][lane] = (re, im): pair-major, so the
// lanes of a warp re-seeding the same pair at different codes read entries
// 32 bytes apart instead of a whole column stride) and seeds
// v0_i = Q_in - sum_{j<n} Q_ij (sV0, [k][lane]), and the +c / -c tables with
// c_ij the double-float rounding of 2 Q_ij 2^-61.  Returns whether any entry
// is non-finite.
template <int N>
__device__ __forceinline__ bool xp_stage_df(const double* __restrict__ A, float4* sP, float4* sM, longlong2* sQ,
                                            longlong2* sV0, int* sG, int* status) {
  constexpr int NP = kPairs<N>;
  if (xp_row_scales<N>(A, sG, status)) return true;
  float* fP = reinterpret_cast<float*>(sP);
  float* fM = reinterpret_cast<float*>(sM);
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const int G = sG[i];
    const int k = i >> 1, lane = i & 1;
    long long q[2], q2[2] = {0, 0};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      q[c] = __double2ll_rn(scalbn(A[(size_t)idx * 2 + c], G + kPdfGrid));
      float h = 0.f, l = 0.f;
      if (j < N - 1) {
        q2[c] = 2 * q[c];
        pdf_split(q2[c], h, l);
      }
      const size_t base = (((size_t)j * NP + k) * 2 + c) * 4;
      fP[base + lane] = h;
      fP[base + 2 + lane] = l;
      fM[base + lane] = -h;
      fM[base + 2 + lane] = -l;
    }
    sQ[((size_t)k * N + j) * 2 + lane] = make_longlong2(q2[0], q2[1]);
    if (j == N - 1) sV0[k * 2 + lane] = make_longlong2(q[0], q[1]);  // Q_in, completed below
  }
  if (N & 1) {
    // the missing row of an odd order: constant 1 (seed 2^61, columns zero)
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const size_t base = (((size_t)j * NP + (NP - 1)) * 2 + c) * 4;
        fP[base + 1] = 0.f, fP[base + 3] = 0.f;
        fM[base + 1] = 0.f, fM[base + 3] = 0.f;
      }
      sQ[((size_t)(NP - 1) * N + j) * 2 + 1] = make_longlong2(0, 0);
    }
    if (threadIdx.x == 0) sV0[(NP - 1) * 2 + 1] = make_longlong2(1ll << kPdfGrid, 0);
  }
  __syncthreads();
  // seeds v0_i = Q_in - sum_{j<n} Q_ij from the int64 table (exact integer sums)
  if (threadIdx.x < N) {
    const int i = threadIdx.x, k = i >> 1, lane = i & 1;
    longlong2 s = sV0[k * 2 + lane];
    for (int j = 0; j < N - 1; ++j) {
      const longlong2 q2 = sQ[((size_t)k * N + j) * 2 + lane];
      s.x -= q2.x >> 1;
      s.y -= q2.y >> 1;
    }
    sV0[k * 2 + lane] = s;
  }
  __syncthreads();
  return false;
}

// Re-seed every row pair from its exact int64 value at code r (App. A steps
// 2, 5-8 in integer form): v_i = v0_i + sum over the set bits j of gray(r) of
// 2 Q_ij, then rounded to a double-float pair.
template <int N>
__device__ __forceinline__ void pdf_seed(P4 (&v)[kPairs<N>], const longlong2* __restrict__ sQ,
                                         const longlong2* __restrict__ sV0, uint64_t r) {
  constexpr int NP = kPairs<N>;
  const uint64_t x0 = r ^ (r >> 1);
  // rows formed in a rolled loop through a per-thread scratch array, so only
  // one pair of int64 row sums is live while it is built
  P4 seed[NP];
#pragma unroll 1
  for (int k = 0; k < NP; ++k) {
    longlong2 a = sV0[2 * k], b = sV0[2 * k + 1];
    uint64_t x = x0;
#pragma unroll 1
    while (x) {
      const int j = __ffsll((long long)x) - 1;
      x &= x - 1;
      const longlong2* q = sQ + ((size_t)k * N + j) * 2;
      const longlong2 qa = q[0], qb = q[1];
      a.x += qa.x;
      a.y += qa.y;
      b.x += qb.x;
      b.y += qb.y;
    }
    P4 t;
    pdf_split(a.x, t.hr.x, t.lr.x);
    pdf_split(b.x, t.hr.y, t.lr.y);
    pdf_split(a.y, t.hi.x, t.li.x);
    pdf_split(b.y, t.hi.y, t.li.y);
    seed[k] = t;
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) v[k] = seed[k];
}

// Per-thread code range: equal lengths rounded up to a multiple of an
// alignment a (2^kXpAlignLog, or the power of two at or above the length when
// that is smaller, so that short launches still use every thread), so every
// thread starts at a code congruent to `first` modulo a.
__device__ __forceinline__ void range_congruent(uint64_t first, uint64_t count, uint64_t T, uint64_t g, uint64_t& r,
                                                uint64_t& end) {
  uint64_t L = (count + T - 1) / T;
  uint64_t kA = 1ull << kXpAlignLog;
  while (kA > 1 && (kA >> 1) >= L) kA >>= 1;
  L = (L + kA - 1) & ~(kA - 1);
  const uint64_t s = g * L;
  r = first + (s < count ? s : count);
  end = first + (s + L < count ? s + L : count);
}

// The whole launch's threads over [first, first + count).
__device__ __forceinline__ void thread_range_congruent(uint64_t first, uint64_t count, uint64_t& r, uint64_t& end) {
  range_congruent(first, count, (uint64_t)gridDim.x * blockDim.x, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                  r, end);
}

// Add one term (-1)^r prod_i u_i, rebuilt as FP64, into the run sums.
template <int N>
__device__ __forceinline__ void xp_term(const P4 (&v)[kPairs<N>], uint32_t odd, double& sr, double& si) {
  cdf z;
  int E;
  xp_product<N>(v, z, E);
  sr += f32_scaled_f64(z.rh, E, odd);
  sr += f32_scaled_f64(z.rl, E, odd);
  si += f32_scaled_f64(z.ih, E, odd);
  si += f32_scaled_f64(z.il, E, odd);
}

// Exact float-pair rows: seeded once, then per code the product, the signed
// accumulation, the Gray step and the exact row update (App. A steps 2-15).
template <int N>
__device__ __forceinline__ void thread_walk_xp_exact(const float4* __restrict__ sP, const float4* __restrict__ sM,
                                                     const float4* __restrict__ sV0, uint64_t r, const uint64_t end,
                                                     dd& accr, dd& acci) {
  constexpr int NP = kPairs<N>;
  if (r >= end) return;
  P4 v[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float4 re = sV0[2 * k], im = sV0[2 * k + 1];
    v[k] = P4{make_float2(re.x, re.y), make_float2(re.z, re.w), make_float2(im.x, im.y), make_float2(im.z, im.w)};
  }
  {
    // seed once (App. A steps 2, 5-8): add the columns of the set bits of gray(r), exactly
    uint64_t x = r ^ (r >> 1);
#pragma unroll 1
    while (x) {
      const int j = __ffsll((long long)x) - 1;
      x &= x - 1;
      const float4* col = sP + (size_t)j * NP * 2;
#pragma unroll
      for (int k = 0; k < NP; ++k) xp_add_col(v[k], col[2 * k], col[2 * k + 1]);
    }
  }
  while (r < end) {
    const uint64_t run_end = min(end, (r | (kRun - 1)) + 1);
    double sr = 0.0, si = 0.0;
    uint32_t odd = (uint32_t)(r & 1ull);
    for (; r < run_end; ++r) {
      xp_term<N>(v, odd, sr, si);
      odd ^= 1u;
      int j;
      uint32_t neg;
      gray_step(r, j, neg);
      const float4* col = (neg ? sM : sP) + (size_t)j * NP * 2;
#pragma unroll
      for (int k = 0; k < NP; ++k) xp_add_col(v[k], col[2 * k], col[2 * k + 1]);
    }
    accr = dd_add_d(accr, sr);
    acci = dd_add_d(acci, si);
  }
}

// Double-float rows: every 2^tile_log codes (counted from the thread's
// start, so the lanes of a warp re-seed together) the rows are re-seeded from
// their exact int64 values; in between, double-float updates.
template <int N>
__device__ __forceinline__ void thread_walk_xp_df(const float4* __restrict__ sP, const float4* __restrict__ sM,
                                                  const longlong2* __restrict__ sQ,
                                                  const longlong2* __restrict__ sV0, uint64_t r, const uint64_t end,
                                                  int tile_log, dd& accr, dd& acci) {
  constexpr int NP = kPairs<N>;
  P4 v[NP];
  while (r < end) {
    const uint64_t tile_end = min(end, r + (uint64_t)(1ull << tile_log));
    pdf_seed<N>(v, sQ, sV0, r);
    double sr = 0.0, si = 0.0;
    uint32_t odd = (uint32_t)(r & 1ull);
    for (; r < tile_end; ++r) {
      xp_term<N>(v, odd, sr, si);
      odd ^= 1u;
      int j;
      uint32_t neg;
      gray_step(r, j, neg);
      const float4* col = (neg ? sM : sP) + (size_t)j * NP * 2;
#pragma unroll
      for (int k = 0; k < NP; ++k) df2_add_col(v[k], col[2 * k], col[2 * k + 1]);
    }
    accr = dd_add_d(accr, sr);
    acci = dd_add_d(acci, si);
  }
}

template <int N, bool EXACT>
__global__ void __launch_bounds__(kWalkThreads) k_walk_xp(const double* __restrict__ A, uint64_t first,
                                                          uint64_t count, double* __restrict__ partials,
                                                          int accumulate, int* __restrict__ status, int tile_log) {
  using Shape = XpShape<N, EXACT>;
  constexpr int NP = kPairs<N>;
  extern __shared__ __align__(16) float4 xsm[];
  float4* sP = xsm;
  float4* sM = sP + Shape::table_f4;
  char* seed = reinterpret_cast<char*>(sM + Shape::table_f4);
  __shared__ int sG[N];
  dd* sRed = reinterpret_cast<dd*>(seed + Shape::seed_bytes);

  bool bad;
  if constexpr (EXACT)
    bad = xp_stage_exact<N>(A, sP, sM, reinterpret_cast<float4*>(seed), sG, status);
  else
    bad = xp_stage_df<N>(A, sP, sM, reinterpret_cast<longlong2*>(seed),
                         reinterpret_cast<longlong2*>(seed) + (size_t)N * NP * 2, sG, status);

  uint64_t r, end;
  thread_range_congruent(first, count, r, end);
  dd accr{0.0, 0.0}, acci{0.0, 0.0};
  if (!bad) {
    if constexpr (EXACT)
      thread_walk_xp_exact<N>(sP, sM, reinterpret_cast<const float4*>(seed), r, end, accr, acci);
    else
      thread_walk_xp_df<N>(sP, sM, reinterpret_cast<const longlong2*>(seed),
                           reinterpret_cast<const longlong2*>(seed) + (size_t)N * NP * 2, r, end, tile_log, accr,
                           acci);
    // prod_i w_i = prod_i u_i 2^(-N - sum_i G_i)   (u_i = 2 w_i 2^G_i)
    int gs = 0;
    for (int i = 0; i < N; ++i) gs += sG[i];
    const int sc = -N - gs;
    accr = dd{scalbn(accr.hi, sc), scalbn(accr.lo, sc)};
    acci = dd{scalbn(acci.hi, sc), scalbn(acci.lo, sc)};
  } else {
    accr = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
    acci = accr;
  }
  __syncthreads();
  block_store<true>(accr, acci, sRed, partials, accumulate);
}

template <int N, bool EXACT>
struct XpKernel {
  static constexpr size_t smem = XpShape<N, EXACT>::smem_bytes;

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
      e = cudaFuncSetAttribute(k_walk_xp<N, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_xp<N, EXACT>, kWalkThreads, smem);
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
    k_walk_xp<N, EXACT><<<a.blocks, kWalkThreads, smem, a.stream>>>(a.A, a.first, a.count, a.partials,
                                                                     a.accumulate, a.status, pdf_tile_log());
    return cudaGetLastError();
  }
};

template <bool EXACT, int LO, int HI>
cudaError_t xp_dispatch(const WalkArgs& a) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    if (a.n == LO) return XpKernel<LO, EXACT>::launch(a);
    return xp_dispatch<EXACT, LO + 1, HI>(a);
  }
}

template <bool EXACT, int LO, int HI>
int xp_blocks_dispatch(int n) {
  if constexpr (LO > HI) {
    return 0;
  } else {
    if (n == LO) return XpKernel<LO, EXACT>::resident_blocks();
    return xp_blocks_dispatch<EXACT, LO + 1, HI>(n);
  }
}

}  // namespace perm

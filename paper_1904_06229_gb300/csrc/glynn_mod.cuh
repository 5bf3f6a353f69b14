// Exact permanents of small-integer matrices modulo four odd moduli < 2^62:
// the Gray-code walk kernel (host entry point in glynn_mod.cu).
//
// The walk is the App. A Gray-code walk with v = 2w (Glynn's form), which is
// an integer for integer A:
//   v_i(x) = 2 a_{i,n} - sum_j a_ij + 2 sum_{j<n, x_j=1} a_ij,
//   2^(n-1) per(A) = (-1)^(n-1) sum_r (-1)^r prod_i v_i(x(r)).
// Row sums are exact int32 (|v_i| <= b_i = sum_j |a_ij| <= 64*127), updated
// by +-2 a_ij per code, so no re-seeding is ever needed.  The product of the
// n row sums is formed exactly over groups of G rows: each half of a group
// in int32, the two halves in one widening multiply to int64.  The groups are
// combined modulo each modulus with Montgomery multiplication (Montgomery
// 1985: REDC with R = 2^64), shared integer work for all four moduli.
//
// Group size: with b = max_i b_i, a group's magnitude is at most b^G.  The
// kernel takes the largest G in {12, 8, 4} with b^G below the smallest
// modulus; then every group is already a residue up to its sign.  If even
// b^4 is not (moduli below about 2^52 with large entries, down to 3), groups
// of 4 are reduced through Montgomery's R^2 step instead: the magnitudes
// (< 2^52) enter REDC against a reduced operand, and the sign is applied to
// the residue.  Each Montgomery product leaves a factor R^-1; the per-thread
// sums are multiplied back once at the end (R^groups, or R^(groups-1) where
// the first group entered through R^2).
//
// Exact sums first: where a per-thread partial sum provably fits in 192 or
// 256 bits (0-1 and +-1 matrices up to n of about 40), the terms are summed
// exactly as multi-limb integers and reduced modulo the moduli once per
// thread, which takes the Montgomery products out of the per-code work.
//
// GB300 note: this path runs on the integer pipes only (IMAD for the
// products), which issue 32x faster than FP64 on this part.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "perm_internal.h"

namespace perm {

constexpr int kModThreads = 128;

// Montgomery product a * b * 2^-64 mod p, for a < p < 2^62 and b < 2^64
// (a * b < p R, so one conditional subtraction suffices).
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t p, uint64_t pinv) {
  const uint64_t tlo = a * b;
  const uint64_t thi = __umul64hi(a, b);
  const uint64_t m = tlo * pinv;
  const uint64_t mphi = __umul64hi(m, p);
  const uint64_t u = thi + mphi + (tlo != 0 ? 1ull : 0ull);
  return u >= p ? u - p : u;
}

// Signed value with |x| < p into [0, p).
__device__ __forceinline__ uint64_t to_residue(int64_t x, uint64_t p) {
  return x < 0 ? (uint64_t)(x + (int64_t)p) : (uint64_t)x;
}

// b^e with saturation at 2^62 (b <= 64 * 127).
__device__ __forceinline__ uint64_t pow_bound(uint64_t b, int e) {
  uint64_t r = 1;
  for (int k = 0; k < e; ++k) {
    if (b != 0 && r > (1ull << 62) / b) return 1ull << 62;
    r *= b;
  }
  return r;
}

// Exact products of the rows in groups of G: each half (G/2 rows) in int32,
// which holds because b^(G/2) < 2^31 whenever b^G < 2^62.
template <int N, int G>
__device__ __forceinline__ void group_products(const int (&v)[N], int64_t (&g)[(N + G - 1) / G]) {
  constexpr int NG = (N + G - 1) / G;
  constexpr int H = G / 2;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    int lo = v[k * G];
#pragma unroll
    for (int m = 1; m < H; ++m)
      if (k * G + m < N) lo *= v[k * G + m];
    if (k * G + H < N) {
      int hi = v[k * G + H];
#pragma unroll
      for (int m = H + 1; m < G; ++m)
        if (k * G + m < N) hi *= v[k * G + m];
      g[k] = (int64_t)lo * (int64_t)hi;
    } else {
      g[k] = lo;
    }
  }
}

// Walk codes [r, end).  SMALLP: the moduli may be smaller than a group.
template <int N, int NP, int G, bool SMALLP>
__device__ __forceinline__ void mod_walk(const int* sA2, const int* sA2m, const int* sV0, uint64_t r, uint64_t end,
                                         const ModConsts& c, uint64_t (&S)[4]) {
  constexpr int NG = (N + G - 1) / G;
  int v[N];
  {
    // seed from the code of r (App. A steps 2, 5-8, with v = 2w)
    const uint64_t x = r ^ (r >> 1);
    int seed[N];
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      int s = sV0[i];
#pragma unroll 1
      for (int j = 0; j < N - 1; ++j) s += ((x >> j) & 1ull) ? sA2[j * NP + i] : 0;
      seed[i] = s;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = seed[i];
  }
  uint32_t odd = (uint32_t)(r & 1ull);
  for (; r < end; ++r) {
    int64_t g[NG];
    group_products<N, G>(v, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t p = c.p[q];
      uint64_t t;
      if constexpr (!SMALLP) {
        t = to_residue(g[0], p);
#pragma unroll
        for (int k = 1; k < NG; ++k) t = mont_mul(t, to_residue(g[k], p), p, c.pinv[q]);
      } else {
        uint32_t neg = g[0] < 0 ? 1u : 0u;
        t = mont_mul(c.r2[q], (uint64_t)(g[0] < 0 ? -g[0] : g[0]), p, c.pinv[q]);
#pragma unroll
        for (int k = 1; k < NG; ++k) {
          neg ^= g[k] < 0 ? 1u : 0u;
          t = mont_mul(t, (uint64_t)(g[k] < 0 ? -g[k] : g[k]), p, c.pinv[q]);
        }
        if (neg && t) t = p - t;
      }
      // (-1)^r term
      const uint64_t add = (odd && t) ? (p - t) : t;
      const uint64_t s = S[q] + add;
      S[q] = s >= p ? s - p : s;
    }
    odd ^= 1u;
    // nextset: column j = ctz(r+1) flips; its new bit is 1 - bit (j+1) of r+1
    const uint64_t r1 = r + 1;
    const int j = __ffsll((long long)r1) - 1;
    const bool neg = (j < 63) && ((r1 >> (j + 1)) & 1ull);
    const int4* col = reinterpret_cast<const int4*>((neg ? sA2m : sA2) + j * NP);
#pragma unroll
    for (int i4 = 0; i4 < NP / 4; ++i4) {
      const int4 d = col[i4];
      if (4 * i4 + 0 < N) v[4 * i4 + 0] += d.x;
      if (4 * i4 + 1 < N) v[4 * i4 + 1] += d.y;
      if (4 * i4 + 2 < N) v[4 * i4 + 2] += d.z;
      if (4 * i4 + 3 < N) v[4 * i4 + 3] += d.w;
    }
  }
  // undo the factors of R left by the Montgomery products
  constexpr int K = SMALLP ? 0 : 1;  // fix[K][q] = R^(NG - 1 + K) mod p for this G
  const int gi = G == 12 ? 0 : (G == 8 ? 1 : 2);
#pragma unroll
  for (int q = 0; q < 4; ++q) S[q] = mont_mul(S[q], c.fix[gi][K][q], c.p[q], c.pinv[q]);
}

// ---- exact integer sums ----
// Where every per-thread partial sum provably fits in L 32-bit limbs, the
// terms are summed exactly (two's complement) and reduced modulo the four
// moduli once per thread.  Each term is the product of ceil(n/H) int32 factors
// (H rows each, |factor| <= b^H < 2^31), built up limb by limb with widening
// 32-bit multiply-adds.

// a += (s ? -x : x), L limbs, as a + (x xor mask) + s with one carry chain.
template <int L>
__device__ __forceinline__ void limbs_add_signed(uint32_t (&a)[L], const uint32_t (&x)[L], uint32_t s);

template <>
__device__ __forceinline__ void limbs_add_signed<6>(uint32_t (&a)[6], const uint32_t (&x)[6], uint32_t s) {
  const uint32_t m = 0u - s;
  asm("{\n\t.reg .u32 t;\n\t"
      "add.cc.u32 t, %6, 0xffffffff;\n\t"
      "addc.cc.u32 %0, %0, %7;\n\t"
      "addc.cc.u32 %1, %1, %8;\n\t"
      "addc.cc.u32 %2, %2, %9;\n\t"
      "addc.cc.u32 %3, %3, %10;\n\t"
      "addc.cc.u32 %4, %4, %11;\n\t"
      "addc.u32 %5, %5, %12;\n\t}"
      : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5])
      : "r"(s), "r"(x[0] ^ m), "r"(x[1] ^ m), "r"(x[2] ^ m), "r"(x[3] ^ m), "r"(x[4] ^ m), "r"(x[5] ^ m));
}

template <>
__device__ __forceinline__ void limbs_add_signed<8>(uint32_t (&a)[8], const uint32_t (&x)[8], uint32_t s) {
  const uint32_t m = 0u - s;
  asm("{\n\t.reg .u32 t;\n\t"
      "add.cc.u32 t, %8, 0xffffffff;\n\t"
      "addc.cc.u32 %0, %0, %9;\n\t"
      "addc.cc.u32 %1, %1, %10;\n\t"
      "addc.cc.u32 %2, %2, %11;\n\t"
      "addc.cc.u32 %3, %3, %12;\n\t"
      "addc.cc.u32 %4, %4, %13;\n\t"
      "addc.cc.u32 %5, %5, %14;\n\t"
      "addc.cc.u32 %6, %6, %15;\n\t"
      "addc.u32 %7, %7, %16;\n\t}"
      : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7])
      : "r"(s), "r"(x[0] ^ m), "r"(x[1] ^ m), "r"(x[2] ^ m), "r"(x[3] ^ m), "r"(x[4] ^ m), "r"(x[5] ^ m),
        "r"(x[6] ^ m), "r"(x[7] ^ m));
}

// Two's-complement L-limb integer -> residue mod p (plain form).
template <int L>
__device__ __forceinline__ uint64_t limbs_mod(const uint32_t (&a)[L], const ModConsts& c, int q) {
  const uint64_t p = c.p[q];
  const bool negative = (a[L - 1] >> 31) != 0;
  uint32_t mag[L];
  uint32_t carry = negative ? 1u : 0u;
#pragma unroll
  for (int w = 0; w < L; ++w) {  // |a| = (a xor mask) + negative
    const uint32_t x = negative ? ~a[w] : a[w];
    mag[w] = x + carry;
    carry = (carry && mag[w] == 0u) ? 1u : 0u;
  }
  uint64_t r = 0;
#pragma unroll
  for (int w = 0; w < L / 2; ++w) {
    const uint64_t word = (uint64_t)mag[2 * w] | ((uint64_t)mag[2 * w + 1] << 32);
    const uint64_t t = mont_mul(c.r2[q], word, p, c.pinv[q]);  // word R mod p
    const uint64_t u = mont_mul(t, c.rpow[w][q], p, c.pinv[q]);  // word R^w mod p
    r += u;
    if (r >= p) r -= p;
  }
  return (negative && r) ? p - r : r;
}

template <int N, int NP, int H, int L>
__device__ __forceinline__ void exact_walk(const int* sA2, const int* sA2m, const int* sV0, uint64_t r, uint64_t end,
                                           const ModConsts& c, uint64_t (&S)[4]) {
  constexpr int NF = (N + H - 1) / H;  // int32 factors per term
  int v[N];
  {
    const uint64_t x = r ^ (r >> 1);
    int seed[N];
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      int s = sV0[i];
#pragma unroll 1
      for (int j = 0; j < N - 1; ++j) s += ((x >> j) & 1ull) ? sA2[j * NP + i] : 0;
      seed[i] = s;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = seed[i];
  }
  uint32_t acc[L];
#pragma unroll
  for (int w = 0; w < L; ++w) acc[w] = 0u;
  uint32_t odd = (uint32_t)(r & 1ull);
  for (; r < end; ++r) {
    uint32_t P[L];
    uint32_t neg = odd;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      int f = v[k * H];
#pragma unroll
      for (int m = 1; m < H; ++m)
        if (k * H + m < N) f *= v[k * H + m];
      neg ^= (uint32_t)f >> 31;
      const uint32_t a = (uint32_t)(f < 0 ? -f : f);
      if (k == 0) {
        P[0] = a;
      } else {
        uint64_t carry = 0;
#pragma unroll
        for (int w = 0; w < (k < L ? k : L); ++w) {
          const uint64_t t = (uint64_t)P[w] * a + carry;
          P[w] = (uint32_t)t;
          carry = t >> 32;
        }
        if (k < L) P[k] = (uint32_t)carry;
      }
    }
#pragma unroll
    for (int w = (NF < L ? NF : L); w < L; ++w) P[w] = 0u;
    limbs_add_signed<L>(acc, P, neg);
    odd ^= 1u;
    const uint64_t r1 = r + 1;
    const int j = __ffsll((long long)r1) - 1;
    const bool flip = (j < 63) && ((r1 >> (j + 1)) & 1ull);
    const int4* col = reinterpret_cast<const int4*>((flip ? sA2m : sA2) + j * NP);
#pragma unroll
    for (int i4 = 0; i4 < NP / 4; ++i4) {
      const int4 d = col[i4];
      if (4 * i4 + 0 < N) v[4 * i4 + 0] += d.x;
      if (4 * i4 + 1 < N) v[4 * i4 + 1] += d.y;
      if (4 * i4 + 2 < N) v[4 * i4 + 2] += d.z;
      if (4 * i4 + 3 < N) v[4 * i4 + 3] += d.w;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) S[q] = limbs_mod<L>(acc, c, q);
}

// Largest order for which the exact-sum walk is compiled (beyond it the
// sums of 0-1 matrices no longer fit in 256 bits).
constexpr int kExactNMax = 48;

template <int N>
__global__ void __launch_bounds__(kModThreads) k_mod(const int8_t* __restrict__ A, ModConsts c, uint64_t count,
                                                     uint64_t* __restrict__ partials) {
  // Column stride: whole int4 loads, and an odd number of 16-byte units, so
  // that when the lanes of a warp do read different columns (the few steps
  // where their Gray codes differ), those start in different banks.
  constexpr int NP = (((N + 3) & ~3) / 4) % 2 == 1 ? ((N + 3) & ~3) : ((N + 3) & ~3) + 4;
  __shared__ __align__(16) int sA2[N * NP];   // +2 a_ij, column-major
  __shared__ __align__(16) int sA2m[N * NP];  // -2 a_ij
  __shared__ int sV0[N];                      // 2 a_{i,n} - sum_j a_ij
  __shared__ int sMax;
  __shared__ double sLog[N];  // log2 max(b_i, 1)
  __shared__ uint64_t sRed[4 * (kModThreads / 32)];
  if (threadIdx.x == 0) sMax = 0;
  for (int idx = threadIdx.x; idx < N * NP; idx += blockDim.x) {
    const int j = idx / NP, i = idx - j * NP;
    const int a2 = i < N ? 2 * (int)A[(size_t)i * N + j] : 0;
    sA2[idx] = a2;
    sA2m[idx] = -a2;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
    int s = 0, sa = 0;
    for (int j = 0; j < N; ++j) {
      const int a = (int)A[(size_t)i * N + j];
      s += a;
      sa += a < 0 ? -a : a;
    }
    sV0[i] = 2 * (int)A[(size_t)i * N + N - 1] - s;
    sLog[i] = log2((double)(sa > 1 ? sa : 1));
    atomicMax(&sMax, sa);
  }
  __syncthreads();
  // |v_i| <= b_i = sum_j |a_ij| <= b = max_i b_i
  const uint64_t b = (uint64_t)sMax;
  // Per-thread ranges of equal length L, rounded up to a multiple of an
  // alignment a (256, or the power of two at or above the length when that is
  // smaller), so all threads start at codes congruent modulo a: the lanes of
  // a warp then flip the same column with the same sign on all but a few
  // steps in a, and the column read is a shared-memory broadcast.
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t L = (count + T - 1) / T;
  uint64_t align = 256;
  while (align > 1 && (align >> 1) >= L) align >>= 1;
  L = (L + align - 1) & ~(align - 1);
  const uint64_t s0 = gid * L;
  const uint64_t r = s0 < count ? s0 : count;
  const uint64_t end = s0 + L < count ? s0 + L : count;

  // Exact sums: every partial sum of a thread is below (L + 1) prod_i b_i;
  // bits = log2 of that bound, plus the sign and a margin for rounding of the
  // logarithms (fixed summation order, the same in every thread).
  double lg = log2((double)(L + 1));
  for (int i = 0; i < N; ++i) lg += sLog[i];
  const int bits = (int)ceil(lg) + 2;
  const int hsix = pow_bound(b, 6) < (1ull << 31);  // factors of 6 rows fit in int32
  int path;
  if (N <= kExactNMax && c.exact_ok && bits <= 192)
    path = hsix ? 4 : 5;
  else if (N <= kExactNMax && c.exact_ok && bits <= 256)
    path = hsix ? 6 : 7;
  else  // modular: the largest group with b^G below every modulus
    path = pow_bound(b, 12) < c.pmin ? 0 : (pow_bound(b, 8) < c.pmin ? 1 : (pow_bound(b, 4) < c.pmin ? 2 : 3));

  uint64_t S[4] = {0, 0, 0, 0};
  if constexpr (N <= kExactNMax) {
    if (path == 4)
      exact_walk<N, NP, 6, 6>(sA2, sA2m, sV0, r, end, c, S);
    else if (path == 5)
      exact_walk<N, NP, 2, 6>(sA2, sA2m, sV0, r, end, c, S);
    else if (path == 6)
      exact_walk<N, NP, 6, 8>(sA2, sA2m, sV0, r, end, c, S);
    else if (path == 7)
      exact_walk<N, NP, 2, 8>(sA2, sA2m, sV0, r, end, c, S);
  }
  if (path == 0)
    mod_walk<N, NP, 12, false>(sA2, sA2m, sV0, r, end, c, S);
  else if (path == 1)
    mod_walk<N, NP, 8, false>(sA2, sA2m, sV0, r, end, c, S);
  else if (path == 2)
    mod_walk<N, NP, 4, false>(sA2, sA2m, sV0, r, end, c, S);
  else if (path == 3)
    mod_walk<N, NP, 4, true>(sA2, sA2m, sV0, r, end, c, S);

  // exact modular sums: any order gives the same residues
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint64_t s = S[q];
    for (int m = 16; m >= 1; m >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, s, m);
      s += o;
      if (s >= c.p[q]) s -= c.p[q];
    }
    S[q] = s;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int q = 0; q < 4; ++q) sRed[warp * 4 + q] = S[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    const int q = threadIdx.x;
    uint64_t s = 0;
    for (int w = 0; w < kModThreads / 32; ++w) {
      s += sRed[w * 4 + q];
      if (s >= c.p[q]) s -= c.p[q];
    }
    partials[(size_t)blockIdx.x * 4 + q] = s;
  }
}

template <int N>
struct ModKernel {
  static int resident() {
    int dev = 0, per_sm = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mod<N>, kModThreads, 0) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return (per_sm < 1 ? 1 : per_sm) * sms;
  }
  static cudaError_t launch(const int8_t* A, const ModConsts& c, uint64_t count, uint64_t* partials, int blocks,
                            cudaStream_t s) {
    k_mod<N><<<blocks, kModThreads, 0, s>>>(A, c, count, partials);
    return cudaGetLastError();
  }
};

template <int LO, int HI>
int mod_resident_dispatch(int n) {
  if constexpr (LO > HI) {
    return 0;
  } else {
    if (n == LO) return ModKernel<LO>::resident();
    return mod_resident_dispatch<LO + 1, HI>(n);
  }
}

template <int LO, int HI>
cudaError_t mod_launch_dispatch(int n, const int8_t* A, const ModConsts& c, uint64_t count, uint64_t* partials,
                                int blocks, cudaStream_t s) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    if (n == LO) return ModKernel<LO>::launch(A, c, count, partials, blocks, s);
    return mod_launch_dispatch<LO + 1, HI>(n, A, c, count, partials, blocks, s);
  }
}

}  // namespace perm

// Exact permanents of small-integer matrices modulo four odd primes < 2^62.
//
// The walk is the App. A Gray-code walk with v = 2w (Glynn's form), which is
// an integer for integer A:
//   v_i(x) = 2 a_{i,n} - sum_j a_ij + 2 sum_{j<n, x_j=1} a_ij,
//   2^(n-1) per(A) = (-1)^(n-1) sum_r (-1)^r prod_i v_i(x(r)).
// Row sums are exact int32 (|v_i| <= sum_j |a_ij| <= 64*127), updated by
// +-2 a_ij per code, so no re-seeding is ever needed.  The product of the n
// row sums is formed exactly in int64 over groups of G rows (G = 8 when every
// |v_i| < 128, else 4; |group| < 2^56 < p either way), and the groups are
// combined modulo each prime with Montgomery multiplication (Montgomery 1985:
// REDC with R = 2^64).  Each Montgomery product leaves a factor R^-1; the
// per-thread sums are multiplied back by R^(groups-1) once at the end.
//
// GB300 note: this path runs on the integer pipes only (IMAD for the 64-bit
// products), which issue 32x faster than FP64 on this part; the exact int64
// grouping replaces most of the n-1 modular multiplications per term and
// prime by single IMADs shared by all four primes.
#include <cuda_runtime.h>

#include <cstdint>

#include "modular_host.h"
#include "perm.h"
#include "perm_internal.h"

namespace perm {

constexpr int kModThreads = 128;

struct ModConsts {
  uint64_t p[4];
  uint64_t pinv[4];  // -p^-1 mod 2^64
  uint64_t fix8[4];  // R^(ceil(N/8)) mod p
  uint64_t fix4[4];  // R^(ceil(N/4)) mod p
};

// Montgomery product a * b * 2^-64 mod p, for a, b < p < 2^62.
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t p, uint64_t pinv) {
  const uint64_t tlo = a * b;
  const uint64_t thi = __umul64hi(a, b);
  const uint64_t m = tlo * pinv;
  const uint64_t mphi = __umul64hi(m, p);
  uint64_t u = thi + mphi + (tlo != 0 ? 1ull : 0ull);
  return u >= p ? u - p : u;
}

// Signed value with |x| < p into [0, p).
__device__ __forceinline__ uint64_t to_residue(int64_t x, uint64_t p) {
  return x < 0 ? (uint64_t)(x + (int64_t)p) : (uint64_t)x;
}

template <int N, int G>
__device__ __forceinline__ void mod_walk(const int* sA2, const int* sV0, uint64_t r, uint64_t end, const ModConsts& c,
                                         uint64_t (&S)[4]) {
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
      for (int j = 0; j < N - 1; ++j) s += ((x >> j) & 1ull) ? sA2[j * N + i] : 0;
      seed[i] = s;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = seed[i];
  }
  uint32_t odd = (uint32_t)(r & 1ull);
  for (; r < end; ++r) {
    int64_t g[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      int64_t t = v[k * G];
#pragma unroll
      for (int m = 1; m < G; ++m)
        if (k * G + m < N) t *= (int64_t)v[k * G + m];
      g[k] = t;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t p = c.p[q];
      uint64_t t = to_residue(g[0], p);
#pragma unroll
      for (int k = 1; k < NG; ++k) t = mont_mul(t, to_residue(g[k], p), p, c.pinv[q]);
      // (-1)^r term
      uint64_t add = odd ? (p - t) : t;
      uint64_t s = S[q] + add;
      S[q] = s >= p ? s - p : s;
    }
    odd ^= 1u;
    // nextset: column j = ctz(r+1) flips; its new bit is 1 - bit (j+1) of r+1
    const uint64_t r1 = r + 1;
    const int j = __ffsll((long long)r1) - 1;
    const bool neg = (j < 63) && ((r1 >> (j + 1)) & 1ull);
    const int* col = sA2 + j * N;
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] += neg ? -col[i] : col[i];
  }
  // undo the R^-(NG-1) left by the Montgomery products
#pragma unroll
  for (int q = 0; q < 4; ++q) S[q] = mont_mul(S[q], G == 8 ? c.fix8[q] : c.fix4[q], c.p[q], c.pinv[q]);
}

template <int N>
__global__ void __launch_bounds__(kModThreads) k_mod(const int8_t* __restrict__ A, ModConsts c, uint64_t count,
                                                     uint64_t* __restrict__ partials) {
  __shared__ int sA2[N * N];  // 2 a_ij, column-major
  __shared__ int sV0[N];      // 2 a_{i,n} - sum_j a_ij
  __shared__ uint64_t sRed[4 * (kModThreads / 32)];
  int rowabs_max = 0;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    sA2[j * N + i] = 2 * (int)A[idx];
  }
  __syncthreads();
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
    int s = 0, sa = 0;
    for (int j = 0; j < N; ++j) {
      const int a = sA2[j * N + i] / 2;
      s += a;
      sa += a < 0 ? -a : a;
    }
    sV0[i] = sA2[(N - 1) * N + i] - s;
    rowabs_max = sa;
  }
  // |v_i| <= sum_j |a_ij|: groups of 8 stay below 2^56 when that is < 128
  const int small = !__syncthreads_or(rowabs_max >= 128);

  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t q0 = count / T, rem = count % T;
  const uint64_t r = gid * q0 + (gid < rem ? gid : rem);
  const uint64_t end = r + q0 + (gid < rem ? 1 : 0);

  uint64_t S[4] = {0, 0, 0, 0};
  if (small)
    mod_walk<N, 8>(sA2, sV0, r, end, c, S);
  else
    mod_walk<N, 4>(sA2, sV0, r, end, c, S);

  // exact modular sums: any order gives the same residues
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint64_t s = S[q];
    for (int m = 16; m >= 1; m >>= 1) {
      uint64_t o = __shfl_xor_sync(0xffffffffu, s, m);
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

// Sum the block residues and multiply by scale_R[q] / R = (-1)^(n-1) 2^-(n-1).
__global__ void k_mod_finalize(const uint64_t* __restrict__ partials, int nparts, ModConsts c, const uint64_t scaleR0,
                               const uint64_t scaleR1, const uint64_t scaleR2, const uint64_t scaleR3,
                               uint64_t* __restrict__ residues) {
  const int q = threadIdx.x;
  if (q >= 4) return;
  const uint64_t p = c.p[q];
  uint64_t s = 0;
  for (int k = 0; k < nparts; ++k) {
    s += partials[(size_t)k * 4 + q];
    if (s >= p) s -= p;
  }
  const uint64_t sr[4] = {scaleR0, scaleR1, scaleR2, scaleR3};
  residues[q] = mont_mul(s, sr[q], p, c.pinv[q]);
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

namespace {

bool is_device_ptr_mod(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

uint64_t pow_r_mod(uint64_t p, int k) {  // R^k mod p, R = 2^64
  uint64_t r = perm::mont_r_mod(p), out = 1 % p;
  for (int i = 0; i < k; ++i) out = perm::mulmod_u64(out, r, p);
  return out;
}

}  // namespace

extern "C" int perm_mod01(const int8_t* A, int n, const uint64_t* primes, uint64_t* residues, void* stream) {
  using namespace perm;
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
  if (!A || !primes || !residues) return PERM_ENULL;
  int rc = check_moduli(primes, 4);
  if (rc) return rc;
  int count_dev = 0, dev = 0;
  if (cudaGetDeviceCount(&count_dev) != cudaSuccess || count_dev < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) return PERM_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;

  ModConsts c;
  uint64_t scaleR[4];
  const int ng8 = (n + 7) / 8, ng4 = (n + 3) / 4;
  for (int q = 0; q < 4; ++q) {
    const uint64_t p = primes[q];
    c.p[q] = p;
    c.pinv[q] = mont_neg_inv(p);
    c.fix8[q] = pow_r_mod(p, ng8);
    c.fix4[q] = pow_r_mod(p, ng4);
    // (-1)^(n-1) / 2^(n-1) mod p, times R for the Montgomery product
    uint64_t inv2 = (p + 1) / 2;
    uint64_t sc = powmod_u64(inv2, (uint64_t)(n - 1), p);
    if (((n - 1) & 1) && sc) sc = p - sc;
    scaleR[q] = mulmod_u64(sc, mont_r_mod(p), p);
  }

  const uint64_t total = 1ull << (n - 1);
  int resident = mod_resident_dispatch<1, PERM_NMAX>(n);
  if (resident < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  const uint64_t per_block = 16ull * kModThreads;
  uint64_t want = (total + per_block - 1) / per_block;
  int blocks = (int)(want < 1 ? 1 : (want > (uint64_t)resident ? (uint64_t)resident : want));

  const bool a_dev = is_device_ptr_mod(A);
  const bool o_dev = is_device_ptr_mod(residues);
  const size_t szA = a_dev ? 0 : (((size_t)n * n + 255) & ~(size_t)255);
  const size_t szP = (((size_t)blocks * 4 * sizeof(uint64_t)) + 255) & ~(size_t)255;
  const size_t szO = o_dev ? 0 : 256;
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, szA + szP + szO, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PERM_ENOMEM : PERM_ECUDA;
  }
  const int8_t* dA = A;
  if (!a_dev) {
    e = cudaMemcpyAsync(base, A, (size_t)n * n, cudaMemcpyHostToDevice, s);
    dA = (const int8_t*)base;
  }
  uint64_t* partials = (uint64_t*)(base + szA);
  uint64_t* dOut = o_dev ? residues : (uint64_t*)(base + szA + szP);
  if (e == cudaSuccess) e = mod_launch_dispatch<1, PERM_NMAX>(n, dA, c, total, partials, blocks, s);
  if (e == cudaSuccess) {
    k_mod_finalize<<<1, 32, 0, s>>>(partials, blocks, c, scaleR[0], scaleR[1], scaleR[2], scaleR[3], dOut);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !o_dev) e = cudaMemcpyAsync(residues, dOut, 4 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(base, s);
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

// Permanents of matrices with repeated columns by the weighted form of
// Ryser's formula, Eq.(ryser2) of Sec. 2.A:
//
//   per(A) = (-1)^n sum_{0 <= f_k <= m_k} (-1)^{sum_k f_k} (prod_k binom(m_k, f_k))
//            prod_i sum_k f_k cbar_k(i)
//
// where A has R distinct columns cbar_k, column k repeated m_k times.  The
// sum has prod_k (m_k + 1) terms instead of 2^(n-1).
//
// Walk: each thread takes a contiguous range of the mixed-radix counting
// index of f (digit 0 fastest) and keeps the row sums s_i = sum_k f_k cbar_k(i)
// as exact int64 fixed point (per-row power-of-two scale, as in the
// fixed-point Gray walk): stepping digit 0 adds C_0, a carry subtracts
// m_k C_k and adds C_{k+1}; none of this rounds, so nothing drifts however
// often carries happen.  The weight is exact table values: binom(m_0, f_0)
// times the product over the other digits, which changes only on a carry.
// The signed weight multiplies the FP64 product, and every term is added
// into double-double accumulators (Eq. ryser2 cancels much more than the
// halved Gray sum does).
#include <cuda_runtime.h>

#include <cstdint>

#include "dd.cuh"
#include "glynn_walk.cuh"
#include "glynn_walk_fx.cuh"
#include "perm.h"
#include "perm_internal.h"

namespace perm {

constexpr int kR2MaxR = PERM_NMAX;

struct R2Params {
  int R;
  int mult[kR2MaxR];
  int bin_off[kR2MaxR];  // offset of column k's binomial row in the table
};

template <int N>
struct R2Shape {
  // +C_k and m_k C_k (int64 pairs, R columns), binomials (<= 2N + R doubles),
  // row exponent biases and scales, reduction slots
  static size_t smem(int R, int nbin) {
    return (size_t)2 * R * N * sizeof(longlong2) + (size_t)nbin * sizeof(double) + 2 * N * sizeof(int) +
           8 * sizeof(dd) + 16;
  }
};

template <int N>
__global__ void __launch_bounds__(kWalkThreads) k_ryser2(const double* __restrict__ Cg, R2Params prm, int nbin,
                                                         uint64_t total, double* __restrict__ partials,
                                                         int* __restrict__ status) {
  extern __shared__ __align__(16) long long r2sm[];
  const int R = prm.R;
  longlong2* sCp = reinterpret_cast<longlong2*>(r2sm);  // [k * N + i] = C_ik
  longlong2* sCm = sCp + R * N;                          // [k * N + i] = m_k C_ik
  double* sBin = reinterpret_cast<double*>(sCm + R * N);
  int* sEb = reinterpret_cast<int*>(sBin + nbin);
  int* sF = sEb + N;
  dd* sRed = reinterpret_cast<dd*>(r2sm);  // reused after the walk

  const double2* C = reinterpret_cast<const double2*>(Cg);  // n x R row-major
  // ---- stage: per-row scales (|s_i| <= sum_k m_k |cbar_k(i)|), tables, binomials
  int bad = 0;
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
    double ar = 0.0, ai = 0.0;
    for (int k = 0; k < R; ++k) {
      const double2 v = C[i * R + k];
      bad |= (not_finite(v.x) || not_finite(v.y)) ? 1 : 0;
      ar += prm.mult[k] * fabs(v.x);
      ai += prm.mult[k] * fabs(v.y);
    }
    const double mx = fmax(ar, ai);
    int F = 0;
    if (mx > 0.0 && !bad) {
      const int ex = dexp_of(mx);
      F = ex == 0 ? 61 + 1022 : 61 - (ex - 1023);
    }
    sF[i] = F;
    sEb[i] = 1086 - F;
  }
  const bool any_bad = __syncthreads_or(bad) != 0;
  if (any_bad && threadIdx.x == 0) atomicOr(status, (int)kStatusNonFinite);
  if (!any_bad) {
    for (int idx = threadIdx.x; idx < N * R; idx += blockDim.x) {
      const int i = idx / R, k = idx - i * R;
      const double2 v = C[idx];
      const int F = sF[i];
      const long long qr = __double2ll_rn(scalbn(v.x, F)), qi = __double2ll_rn(scalbn(v.y, F));
      sCp[k * N + i] = make_longlong2(qr, qi);
      sCm[k * N + i] = make_longlong2((long long)prm.mult[k] * qr, (long long)prm.mult[k] * qi);
    }
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
      // binom(m, f) for f = 0..m by the multiplicative recurrence (exact while < 2^53)
      const int m = prm.mult[k];
      double b = 1.0;
      sBin[prm.bin_off[k]] = 1.0;
      for (int f = 1; f <= m; ++f) {
        b = b * (double)(m - f + 1) / (double)f;
        sBin[prm.bin_off[k] + f] = b;
      }
    }
  }
  __syncthreads();

  uint64_t r, end;
  thread_range(0, total, r, end);
  dd accr{0.0, 0.0}, acci{0.0, 0.0};
  if (any_bad) {
    accr = acci = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
  } else if (r < end) {
    const double z = sBin[0] * 0.0;  // register zero for the product FMAs
    // ---- seed: digits of r, row sums from scratch, weight of the upper digits
    int f[kR2MaxR];
    {
      uint64_t q = r;
#pragma unroll 1
      for (int k = 0; k < R; ++k) {
        const uint64_t rad = (uint64_t)prm.mult[k] + 1;
        f[k] = (int)(q % rad);
        q /= rad;
      }
    }
    long long vr[N], vi[N];
    {
      longlong2 seed[N];
#pragma unroll 1
      for (int i = 0; i < N; ++i) {
        long long sr = 0, si = 0;
#pragma unroll 1
        for (int k = 0; k < R; ++k) {
          const longlong2 c = sCp[k * N + i];
          sr += (long long)f[k] * c.x;
          si += (long long)f[k] * c.y;
        }
        seed[i] = make_longlong2(sr, si);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        vr[i] = seed[i].x;
        vi[i] = seed[i].y;
      }
    }
    const int m0 = prm.mult[0];
    const double* bin0 = sBin;  // bin_off[0] == 0
    int f0 = f[0];
    double wrest = 1.0;
    int par = f0;
#pragma unroll 1
    for (int k = 1; k < R; ++k) wrest *= sBin[prm.bin_off[k] + f[k]], par += f[k];
    uint32_t odd = (uint32_t)(par & 1);
    {
      // Eq.(ryser2) sums terms of both signs and very different sizes (its
      // condition number grows much faster than the halved Gray sum's), so
      // every term goes straight into the double-double accumulators.
      for (; r < end; ++r) {
        double pr, pi;
        FxProduct<N, true, kProdF64>::eval(vr, vi, sEb, pr, pi, z);
        const double sw = flip_sign(fma(wrest, bin0[f0], z), odd);  // (-1)^{sum f} prod binom
        accr = dd_add_d(accr, fma(sw, pr, z));
        acci = dd_add_d(acci, fma(sw, pi, z));
        if (r + 1 >= end) continue;  // no step past this thread's range
        if (f0 < m0) {
          ++f0;
          odd ^= 1u;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const longlong2 c = sCp[i];
            vr[i] += c.x;
            vi[i] += c.y;
          }
        } else {
          // carry: digit 0 back to 0, then every digit at its maximum back to
          // 0, then the next digit up by one
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const longlong2 c = sCm[i];
            vr[i] -= c.x;
            vi[i] -= c.y;
          }
          f0 = 0;
          int k = 1;
          while (k < R && f[k] == prm.mult[k]) {
            const longlong2* cm = sCm + k * N;
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const longlong2 c = cm[i];
              vr[i] -= c.x;
              vi[i] -= c.y;
            }
            f[k] = 0;
            ++k;
          }
          if (k < R) {
            ++f[k];
            const longlong2* cp = sCp + k * N;
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const longlong2 c = cp[i];
              vr[i] += c.x;
              vi[i] += c.y;
            }
          }
          wrest = 1.0;
          par = 0;
#pragma unroll 1
          for (int kk = 1; kk < R; ++kk) wrest *= sBin[prm.bin_off[kk] + f[kk]], par += f[kk];
          odd = (uint32_t)(par & 1);
        }
      }
    }
  }
  __syncthreads();
  block_store<true>(accr, acci, sRed, partials, 0);
}

template <int N>
struct R2Kernel {
  static cudaError_t launch(const double* C, const R2Params& p, int nbin, uint64_t total, double* partials,
                            int blocks, int* status, cudaStream_t s, int* resident_out) {
    const size_t smem = R2Shape<N>::smem(p.R, nbin);
    cudaError_t e = cudaFuncSetAttribute(k_ryser2<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, per_sm = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ryser2<N>, kWalkThreads, smem)) != cudaSuccess)
      return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int resident = (per_sm < 1 ? 1 : per_sm) * sms;
    if (resident_out) {
      *resident_out = resident;
      return cudaSuccess;
    }
    if (blocks > resident) blocks = resident;
    k_ryser2<N><<<blocks, kWalkThreads, smem, s>>>(C, p, nbin, total, partials, status);
    return cudaGetLastError();
  }
};

template <int LO, int HI>
cudaError_t r2_dispatch(int n, const double* C, const R2Params& p, int nbin, uint64_t total, double* partials,
                        int blocks, int* status, cudaStream_t s, int* resident_out) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    if (n == LO) return R2Kernel<LO>::launch(C, p, nbin, total, partials, blocks, status, s, resident_out);
    return r2_dispatch<LO + 1, HI>(n, C, p, nbin, total, partials, blocks, status, s, resident_out);
  }
}

}  // namespace perm

namespace {

bool device_ptr_r2(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int perm_c128_repeated(const double* C, const int* mult, int R, int n, double* out, void* stream) {
  using namespace perm;
  if (n < 1 || n > PERM_NMAX || R < 1 || R > n) return PERM_EINVAL;
  if (!C || !mult || !out) return PERM_ENULL;
  R2Params p{};
  p.R = R;
  int sum = 0, nbin = 0;
  uint64_t total = 1;
  for (int k = 0; k < R; ++k) {
    if (mult[k] < 1) return PERM_EINVAL;
    p.mult[k] = mult[k];
    p.bin_off[k] = nbin;
    nbin += mult[k] + 1;
    sum += mult[k];
    if (total > (1ull << 62) / (uint64_t)(mult[k] + 1)) return PERM_EINVAL;  // more than 2^62 terms
    total *= (uint64_t)(mult[k] + 1);
  }
  if (sum != n) return PERM_EINVAL;
  int ndev = 0, dev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) return PERM_ECUDA;
  int* status = nullptr;
  if (device_status_word(dev, &status) != 0) return PERM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  int resident = 0;
  cudaError_t e = r2_dispatch<1, PERM_NMAX>(n, nullptr, p, nbin, total, nullptr, 0, nullptr, s, &resident);
  if (e != cudaSuccess || resident < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  const uint64_t per_block = 16ull * kWalkThreads;
  uint64_t want = (total + per_block - 1) / per_block;
  const int blocks = (int)(want < 1 ? 1 : (want > (uint64_t)resident ? (uint64_t)resident : want));

  const bool c_dev = device_ptr_r2(C), o_dev = device_ptr_r2(out);
  const size_t szC = c_dev ? 0 : (((size_t)n * R * 16 + 255) & ~(size_t)255);
  const size_t szP = (((size_t)blocks * 32) + 255) & ~(size_t)255;
  const size_t szO = o_dev ? 0 : 256;
  char* base = nullptr;
  e = cudaMallocAsync((void**)&base, szC + szP + szO, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PERM_ENOMEM : PERM_ECUDA;
  }
  const double* dC = C;
  if (!c_dev) {
    e = cudaMemcpyAsync(base, C, (size_t)n * R * 16, cudaMemcpyHostToDevice, s);
    dC = (const double*)base;
  }
  double* partials = (double*)(base + szC);
  double* dOut = o_dev ? out : (double*)(base + szC + szP);
  if (e == cudaSuccess) e = r2_dispatch<1, PERM_NMAX>(n, dC, p, nbin, total, partials, blocks, status, s, nullptr);
  if (e == cudaSuccess) e = finalize_launch(partials, blocks, true, n, 2, dOut, s);
  if (e == cudaSuccess && !o_dev) e = cudaMemcpyAsync(out, dOut, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(base, s);
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

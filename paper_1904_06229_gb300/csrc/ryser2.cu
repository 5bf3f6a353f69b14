// Permanents of matrices with repeated columns: the multiplicity classes of
// Eq.(ryser2), Sec. 2.A.
//
// A has R distinct columns cbar_k, column k repeated m_k times.  Eq.(ryser2)
// groups Ryser's subsets by how many copies of each distinct column they
// hold, so the sum has prod_k (m_k + 1) terms instead of 2^n.  The kernel
// groups the terms of Glynn's halved form the same way -- the form App. A
// uses for general matrices -- because it is far better conditioned (on
// Haar submatrices with 8 doubled columns the un-halved sum's condition
// number is about 1.7e5, the halved one's about 1e2):
//
//   per(A) = 2^(1-n) sum_{g} (-1)^{sum g} C(m_0 - 1, g_0) prod_{k>=1} C(m_k, g_k)
//            prod_i sum_k (m_k - 2 g_k) cbar_k(i),
//
// g_k = how many of column k's copies carry the sign -1 (one copy of column 0
// is fixed to +1, so 0 <= g_0 <= m_0 - 1 and 0 <= g_k <= m_k otherwise):
// m_0 prod_{k>=1} (m_k + 1) terms.  Tests compare it with the oracle's literal
// evaluation of Eq.(ryser2) and with the Gray walk of the expanded matrix.
//
// Walk: each thread takes a contiguous range of the mixed-radix counting
// index of g (digit 0 fastest) and keeps the row sums
// s_i = sum_k (m_k - 2 g_k) cbar_k(i) as exact int64 fixed point (per-row
// power-of-two scale, as in the fixed-point Gray walk): stepping digit k
// subtracts 2 C_k, a carry adds 2 gmax_k C_k back; none of this rounds.  The
// weight is exact table values: C(gmax_0, g_0) times the product over the
// other digits, which changes only on a carry.  The signed weight multiplies
// the product of the row sums, formed as in the fixed-point Gray walk (most
// factors in integer block floating point, the rest in FP64); terms are
// summed like the Gray walk's (FP64 run sums folded into double-double).
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
  int gmax[kR2MaxR];     // m_0 - 1 for column 0, m_k otherwise
  int bin_off[kR2MaxR];  // offset of row C(gmax_k, .) in the binomial table
};

template <int N>
struct R2Shape {
  // 2 C_k (step) and 2 gmax_k C_k (carry) as int64 pairs, R columns; the
  // binomial rows; row exponent biases and scales; reduction slots
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
  longlong2* sStep = reinterpret_cast<longlong2*>(r2sm);  // [k * N + i] = 2 C_ik
  longlong2* sReset = sStep + R * N;                       // [k * N + i] = 2 gmax_k C_ik
  double* sBin = reinterpret_cast<double*>(sReset + R * N);
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
      sStep[k * N + i] = make_longlong2(2 * qr, 2 * qi);
      sReset[k * N + i] = make_longlong2(2 * (long long)prm.gmax[k] * qr, 2 * (long long)prm.gmax[k] * qi);
    }
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
      // C(gm, g) for g = 0..gm by the multiplicative recurrence (exact while < 2^53)
      const int gm = prm.gmax[k];
      double b = 1.0;
      sBin[prm.bin_off[k]] = 1.0;
      for (int g = 1; g <= gm; ++g) {
        b = b * (double)(gm - g + 1) / (double)g;
        sBin[prm.bin_off[k] + g] = b;
      }
    }
  }
  __syncthreads();
  // The products multiply the unscaled row values v_i 2^-63 (below 1 in
  // magnitude, so no chain leaves the double range however the rows are
  // scaled); the rows' scales are applied once, to the thread's sum.
  int scale = 0;
  if (!any_bad) {
    for (int i = 0; i < N; ++i) scale += sEb[i] - 1023;
    __syncthreads();  // every thread has read sEb before it is overwritten
    if (threadIdx.x < N) sEb[threadIdx.x] = 1023;
    __syncthreads();
  }

  uint64_t r, end;
  thread_range(0, total, r, end);
  dd accr{0.0, 0.0}, acci{0.0, 0.0};
  if (any_bad) {
    accr = acci = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
  } else if (r < end) {
    const double z = sBin[0] * 0.0;  // register zero for the product FMAs
    // ---- seed: digits of r, row sums from scratch, weight of the upper digits
    int g[kR2MaxR];
    {
      uint64_t q = r;
#pragma unroll 1
      for (int k = 0; k < R; ++k) {
        const uint64_t rad = (uint64_t)prm.gmax[k] + 1;
        g[k] = (int)(q % rad);
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
          // (m_k - 2 g_k) C_ik = (m_k - 2 g_k) / 2 * (2 C_ik), exact
          const longlong2 c = sStep[k * N + i];
          const long long f = prm.mult[k] - 2 * g[k];
          sr += f * (c.x / 2);
          si += f * (c.y / 2);
        }
        seed[i] = make_longlong2(sr, si);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        vr[i] = seed[i].x;
        vi[i] = seed[i].y;
      }
    }
    const int gmax0 = prm.gmax[0];
    const double* bin0 = sBin;  // bin_off[0] == 0
    int g0 = g[0];
    double wrest = 1.0;
    int par = g0;
#pragma unroll 1
    for (int k = 1; k < R; ++k) wrest *= sBin[prm.bin_off[k] + g[k]], par += g[k];
    uint32_t odd = (uint32_t)(par & 1);
    const int ixc = ix_offset<N>(sEb);
    while (r < end) {
      const uint64_t run_end = min(end, r + kRun);
      double sr = 0.0, si = 0.0;
      for (; r < run_end; ++r) {
        double pr, pi;
        FxProduct<N, true, kProdF64>::eval(vr, vi, sEb, pr, pi, z, ixc);
        const double sw = flip_sign(fma(wrest, bin0[g0], z), odd);  // (-1)^{sum g} prod binom
        sr = fma(sw, pr, sr);
        si = fma(sw, pi, si);
        if (r + 1 >= end) continue;  // no step past this thread's range
        if (g0 < gmax0) {
          ++g0;
          odd ^= 1u;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const longlong2 c = sStep[i];
            vr[i] -= c.x;
            vi[i] -= c.y;
          }
        } else {
          // carry: digit 0 back to 0, then every digit at its maximum back to
          // 0, then the next digit up by one
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const longlong2 c = sReset[i];
            vr[i] += c.x;
            vi[i] += c.y;
          }
          g0 = 0;
          int k = 1;
          while (k < R && g[k] == prm.gmax[k]) {
            const longlong2* cr = sReset + k * N;
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const longlong2 c = cr[i];
              vr[i] += c.x;
              vi[i] += c.y;
            }
            g[k] = 0;
            ++k;
          }
          if (k < R) {
            ++g[k];
            const longlong2* cs = sStep + k * N;
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const longlong2 c = cs[i];
              vr[i] -= c.x;
              vi[i] -= c.y;
            }
          }
          wrest = 1.0;
          par = 0;
#pragma unroll 1
          for (int kk = 1; kk < R; ++kk) wrest *= sBin[prm.bin_off[kk] + g[kk]], par += g[kk];
          odd = (uint32_t)(par & 1);
        }
      }
      accr = dd_add_d(accr, sr);
      acci = dd_add_d(acci, si);
    }
    accr = dd{scalbn(accr.hi, scale), scalbn(accr.lo, scale)};
    acci = dd{scalbn(acci.hi, scale), scalbn(acci.lo, scale)};
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

template <int LO, int HI>
void r2_preload() {
  if constexpr (LO <= HI) {
    load_kernel(k_ryser2<LO>);
    r2_preload<LO + 1, HI>();
  }
}

void preload_ryser2_kernels() { r2_preload<1, PERM_NMAX>(); }

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
  perm::TraceRange trace("perm_c128_repeated");
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
    p.gmax[k] = k == 0 ? mult[k] - 1 : mult[k];
    p.bin_off[k] = nbin;
    nbin += p.gmax[k] + 1;
    sum += mult[k];
    if (total > (1ull << 62) / (uint64_t)(p.gmax[k] + 1)) return PERM_EINVAL;  // more than 2^62 terms
    total *= (uint64_t)(p.gmax[k] + 1);
  }
  if (sum != n) return PERM_EINVAL;
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
  if (e == cudaSuccess) e = finalize_launch(partials, blocks, true, n, 3, dOut, s);
  if (e == cudaSuccess && !o_dev) e = cudaMemcpyAsync(out, dOut, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(base, s);
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

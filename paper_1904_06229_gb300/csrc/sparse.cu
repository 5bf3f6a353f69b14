// Permanents of sparse matrices by Ryser's sum restricted to the sets J that
// can give a non-zero product (Sec. 2.D, App. B "sparsepermanent" and
// "greedypartition").
//
// A product prod_i sum_{j in J} a_ij vanishes unless J meets the non-zero
// columns N_i of every row i.  greedypartition picks rows whose N_i are
// pairwise disjoint (least out-degree first); with S_l those N_i and T the
// remaining columns, every useful J is a non-empty subset of each S_l plus
// any subset of T: 2^|T| prod_l (2^|S_l| - 1) sets instead of 2^n.  The host
// runs the greedy step with several randomised tie-breaks (App. B notes this
// helps) and keeps the partition with the fewest sets.
//
// Walk: the sets are indexed by a mixed-radix counter whose digit 0 runs over
// the subsets of T and digit l over the non-empty subsets of S_l, each digit
// in binary-reflected Gray order, so stepping a digit toggles one column and
// wrapping a digit toggles one (T) or two (S_l) columns.  Row sums are exact
// int64 fixed point (per-row power-of-two scale, as in the fixed-point Gray
// walk), products as in that walk (integer block floating point for most
// factors, FP64 with round-to-nearest conversions for the rest), and each
// signed term is added straight into double-double accumulators (Ryser's
// un-halved sum cancels strongly).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "dd.cuh"
#include "glynn_walk.cuh"
#include "glynn_walk_fx.cuh"
#include "perm.h"
#include "perm_internal.h"

namespace perm {

constexpr int kSpMaxDig = PERM_NMAX + 1;

struct SpParams {
  int ndig;                  // digit 0 = T (possibly empty), digits 1.. = blocks S_l
  int size[kSpMaxDig];       // columns in the digit's set
  int off[kSpMaxDig];        // offset of its columns in col[]
  int col[PERM_NMAX];        // column indices grouped by digit
  uint64_t radix[kSpMaxDig]; // 2^size for T, 2^size - 1 for a block
};

template <int N>
struct SpShape {
  static constexpr int kStride = N + 1;  // padded column stride (fewer bank conflicts)
  static constexpr size_t smem = (size_t)N * kStride * sizeof(longlong2) + 2 * N * sizeof(int) + 8 * sizeof(dd) + 16;
};

// Subset (as a bitmask over the digit's own columns) at position p.
__device__ __forceinline__ uint64_t sp_subset(int k, uint64_t p) {
  const uint64_t g = k == 0 ? p : p + 1;  // blocks skip the empty subset
  return g ^ (g >> 1);
}

template <int N>
__global__ void __launch_bounds__(kWalkThreads) k_sparse(const double* __restrict__ Ag, SpParams prm, uint64_t total,
                                                         double* __restrict__ partials, int* __restrict__ status) {
  constexpr int ST = SpShape<N>::kStride;
  extern __shared__ __align__(16) long long spm[];
  longlong2* sC = reinterpret_cast<longlong2*>(spm);  // [j * ST + i] = rint(a_ij 2^F_i)
  int* sEb = reinterpret_cast<int*>(sC + N * ST);
  int* sF = sEb + N;
  dd* sRed = reinterpret_cast<dd*>(spm);  // reused after the walk
  const double2* A = reinterpret_cast<const double2*>(Ag);

  int bad = 0;
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
    double ar = 0.0, ai = 0.0;
    for (int j = 0; j < N; ++j) {
      const double2 v = A[i * N + j];
      bad |= (not_finite(v.x) || not_finite(v.y)) ? 1 : 0;
      ar += fabs(v.x);
      ai += fabs(v.y);
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
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int i = idx / N, j = idx - i * N;
      const double2 v = A[idx];
      const int F = sF[i];
      sC[j * ST + i] = make_longlong2(__double2ll_rn(scalbn(v.x, F)), __double2ll_rn(scalbn(v.y, F)));
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
    const double z = fx_to_double(sC[0].x, sEb[0]) * 0.0;
    // ---- seed: digit positions of r, the set J, row sums from scratch
    uint64_t pos[kSpMaxDig];
    uint64_t J = 0;
    {
      uint64_t q = r;
#pragma unroll 1
      for (int k = 0; k < prm.ndig; ++k) {
        pos[k] = q % prm.radix[k];
        q /= prm.radix[k];
        const uint64_t sub = sp_subset(k, pos[k]);
#pragma unroll 1
        for (int b = 0; b < prm.size[k]; ++b)
          if ((sub >> b) & 1ull) J |= 1ull << prm.col[prm.off[k] + b];
      }
    }
    long long vr[N], vi[N];
    {
      longlong2 seed[N];
#pragma unroll 1
      for (int i = 0; i < N; ++i) {
        long long sr = 0, si = 0;
#pragma unroll 1
        for (int j = 0; j < N; ++j)
          if ((J >> j) & 1ull) sr += sC[j * ST + i].x, si += sC[j * ST + i].y;
        seed[i] = make_longlong2(sr, si);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        vr[i] = seed[i].x;
        vi[i] = seed[i].y;
      }
    }
    uint32_t odd = (uint32_t)(__popcll((long long)J) & 1);
    const int t0 = prm.size[0];
    const int ixc = ix_offset<N>(sEb);
    for (; r < end; ++r) {
      double pr, pi;
      FxProduct<N, true, kProdF64, true>::eval(vr, vi, sEb, pr, pi, z, ixc);
      accr = dd_add_d(accr, flip_sign(pr, odd));  // (-1)^|J| prod_i s_i
      acci = dd_add_d(acci, flip_sign(pi, odd));
      if (r + 1 >= end) continue;
      // ---- next set: step digit 0, carrying into higher digits on a wrap
      // toggle column c: row sums +- column, J and the sign of (-1)^|J|
      auto toggle = [&](int c) {
        const long long m = ((J >> c) & 1ull) ? -1ll : 0ll;  // in J: subtract
        const longlong2* colp = sC + c * ST;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const longlong2 cv = colp[i];
          vr[i] += (cv.x ^ m) - m;
          vi[i] += (cv.y ^ m) - m;
        }
        J ^= 1ull << c;
        odd ^= 1u;
      };
      if (pos[0] + 1 < prm.radix[0]) {
        // T: gray(p) -> gray(p+1) flips bit ctz(p+1)
        toggle(prm.col[__ffsll((long long)(pos[0] + 1)) - 1]);
        ++pos[0];
      } else {
        if (t0 > 0) toggle(prm.col[t0 - 1]);  // gray(2^t - 1) is the top bit alone
        pos[0] = 0;
#pragma unroll 1
        for (int k = 1; k < prm.ndig; ++k) {
          const int sz = prm.size[k], o = prm.off[k];
          if (pos[k] + 1 < prm.radix[k]) {
            // block position p holds gray(p+1); p -> p+1 flips bit ctz(p+2)
            toggle(prm.col[o + __ffsll((long long)(pos[k] + 2)) - 1]);
            ++pos[k];
            break;
          }
          if (sz > 1) {  // gray(2^s - 1) (top bit) back to gray(1) (bit 0)
            toggle(prm.col[o + sz - 1]);
            toggle(prm.col[o]);
          }
          pos[k] = 0;
        }
      }
    }
    accr = dd{scalbn(accr.hi, scale), scalbn(accr.lo, scale)};
    acci = dd{scalbn(acci.hi, scale), scalbn(acci.lo, scale)};
  }
  __syncthreads();
  block_store<true>(accr, acci, sRed, partials, 0);
}

template <int N>
struct SpKernel {
  static cudaError_t run(const double* A, const SpParams& p, uint64_t total, double* partials, int blocks, int* status,
                         cudaStream_t s, int* resident_out) {
    const size_t smem = SpShape<N>::smem;
    cudaError_t e = cudaFuncSetAttribute(k_sparse<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, per_sm = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sparse<N>, kWalkThreads, smem)) != cudaSuccess)
      return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int resident = (per_sm < 1 ? 1 : per_sm) * sms;
    if (resident_out) {
      *resident_out = resident;
      return cudaSuccess;
    }
    if (blocks > resident) blocks = resident;
    k_sparse<N><<<blocks, kWalkThreads, smem, s>>>(A, p, total, partials, status);
    return cudaGetLastError();
  }
};

template <int LO, int HI>
cudaError_t sp_dispatch(int n, const double* A, const SpParams& p, uint64_t total, double* partials, int blocks,
                        int* status, cudaStream_t s, int* resident_out) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    if (n == LO) return SpKernel<LO>::run(A, p, total, partials, blocks, status, s, resident_out);
    return sp_dispatch<LO + 1, HI>(n, A, p, total, partials, blocks, status, s, resident_out);
  }
}

template <int LO, int HI>
void sp_preload() {
  if constexpr (LO <= HI) {
    load_kernel(k_sparse<LO>);
    sp_preload<LO + 1, HI>();
  }
}

void preload_sparse_kernels() { sp_preload<1, PERM_NMAX>(); }

}  // namespace perm

namespace {

// greedypartition (App. B) on the non-zero pattern; `rand_state` == 0 takes
// the first least-degree row, otherwise ties are broken by an LCG stream.
void greedy_once(const std::vector<uint8_t>& nz, int n, uint64_t rand_state, std::vector<int>& block) {
  std::vector<int> deg(n, 0);
  std::vector<uint64_t> nbr(n, 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (nz[(size_t)i * n + j]) ++deg[i], nbr[i] |= 1ull << j;
  uint64_t V = n == 64 ? ~0ull : ((1ull << n) - 1);
  block.assign(n, -1);
  int d = 0;
  while (V) {
    int dmin = n + 1;
    for (int i = 0; i < n; ++i)
      if ((V >> i) & 1ull) dmin = std::min(dmin, deg[i]);
    std::vector<int> cand;
    for (int i = 0; i < n; ++i)
      if (((V >> i) & 1ull) && deg[i] == dmin) cand.push_back(i);
    int k = cand[0];
    if (rand_state) {
      rand_state = rand_state * 6364136223846793005ull + 1442695040888963407ull;
      k = cand[(size_t)((rand_state >> 33) % cand.size())];
    }
    const uint64_t Nk = nbr[k];
    for (int j = 0; j < n; ++j)
      if ((Nk >> j) & 1ull) block[j] = d;
    ++d;
    V &= ~(1ull << k);
    for (int l = 0; l < n; ++l)
      if (((V >> l) & 1ull) && (nbr[l] & Nk)) V &= ~(1ull << l);
  }
}

// log2 of the number of sets, and the exact count when it is below 2^63.
double count_log2(const std::vector<int>& block, int n, uint64_t* exact) {
  std::vector<int> sz(n + 1, 0);
  int t = 0, d = 0;
  for (int j = 0; j < n; ++j) {
    if (block[j] < 0)
      ++t;
    else
      ++sz[block[j]], d = std::max(d, block[j] + 1);
  }
  double lg = t;
  unsigned __int128 c = (unsigned __int128)1 << t;
  bool big = t >= 63;
  for (int l = 0; l < d; ++l) {
    lg += std::log2((double)((1ull << sz[l]) - 1));
    c *= (unsigned __int128)((1ull << sz[l]) - 1);
    if (c >= ((unsigned __int128)1 << 63)) big = true;
  }
  *exact = big ? 0 : (uint64_t)c;
  return lg;
}

int best_partition(const std::vector<uint8_t>& nz, int n, int restarts, std::vector<int>& best, uint64_t* count) {
  double best_lg = 1e30;
  std::vector<int> b;
  for (int rs = 0; rs < restarts; ++rs) {
    greedy_once(nz, n, rs == 0 ? 0 : 0x9E3779B97F4A7C15ull * (uint64_t)rs + 1, b);
    uint64_t c = 0;
    const double lg = count_log2(b, n, &c);
    if (lg < best_lg) best_lg = lg, best = b, *count = c;
  }
  return *count ? PERM_OK : PERM_EINVAL;
}

bool device_ptr_sp(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

constexpr int kRestarts = 16;

}  // namespace

extern "C" {

int perm_sparse_partition(const double* A_host, int n, int* block, uint64_t* count) {
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
  if (!A_host || !block || !count) return PERM_ENULL;
  std::vector<uint8_t> nz((size_t)n * n);
  for (size_t e = 0; e < (size_t)n * n; ++e) nz[e] = (A_host[2 * e] != 0.0 || A_host[2 * e + 1] != 0.0);
  std::vector<int> b;
  uint64_t c = 0;
  int rc = best_partition(nz, n, kRestarts, b, &c);
  std::memcpy(block, b.data(), sizeof(int) * n);
  *count = c;
  return rc;
}

int perm_c128_sparse(const double* A, int n, double* out, void* stream) {
  using namespace perm;
  TraceRange trace("perm_c128_sparse");
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
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
  const size_t bytesA = (size_t)n * n * 16;
  const bool a_dev = device_ptr_sp(A), o_dev = device_ptr_sp(out);
  // the partition needs the non-zero pattern on the host
  std::vector<double> hA((size_t)2 * n * n);
  if (a_dev) {
    if (cudaMemcpyAsync(hA.data(), A, bytesA, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PERM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
  } else {
    std::memcpy(hA.data(), A, bytesA);
  }
  int block[PERM_NMAX];
  uint64_t total = 0;
  int rc = perm_sparse_partition(hA.data(), n, block, &total);
  if (rc) return rc;  // more than 2^63 sets
  SpParams p{};
  {
    int d = 0;
    for (int j = 0; j < n; ++j) d = std::max(d, block[j] + 1);
    p.ndig = d + 1;
    int o = 0;
    for (int k = 0; k < p.ndig; ++k) {
      const int want = k == 0 ? -1 : k - 1;
      p.off[k] = o;
      p.size[k] = 0;
      for (int j = 0; j < n; ++j)
        if (block[j] == want) p.col[o++] = j, ++p.size[k];
      p.radix[k] = k == 0 ? (1ull << p.size[k]) : ((1ull << p.size[k]) - 1);
    }
  }
  int resident = 0;
  cudaError_t e = sp_dispatch<1, PERM_NMAX>(n, nullptr, p, total, nullptr, 0, nullptr, s, &resident);
  if (e != cudaSuccess || resident < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  const uint64_t per_block = 16ull * kWalkThreads;
  uint64_t want = (total + per_block - 1) / per_block;
  const int blocks = (int)(want < 1 ? 1 : (want > (uint64_t)resident ? (uint64_t)resident : want));
  const size_t szA = a_dev ? 0 : ((bytesA + 255) & ~(size_t)255);
  const size_t szP = (((size_t)blocks * 32) + 255) & ~(size_t)255;
  const size_t szO = o_dev ? 0 : 256;
  char* base = nullptr;
  e = cudaMallocAsync((void**)&base, szA + szP + szO, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PERM_ENOMEM : PERM_ECUDA;
  }
  const double* dA = A;
  if (!a_dev) {
    e = cudaMemcpyAsync(base, A, bytesA, cudaMemcpyHostToDevice, s);
    dA = (const double*)base;
  }
  double* partials = (double*)(base + szA);
  double* dOut = o_dev ? out : (double*)(base + szA + szP);
  if (e == cudaSuccess) e = sp_dispatch<1, PERM_NMAX>(n, dA, p, total, partials, blocks, status, s, nullptr);
  if (e == cudaSuccess) e = finalize_launch(partials, blocks, true, n, 2, dOut, s);
  if (e == cudaSuccess && !o_dev) e = cudaMemcpyAsync(out, dOut, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(base, s);
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

}  // extern "C"

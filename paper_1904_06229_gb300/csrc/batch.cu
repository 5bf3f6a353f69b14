// Batched permanents: many independent complex matrices of uneven order in
// one graph launch (the random-matrix studies of Secs. 3-6 compute
// 10^5..10^7 permanents of orders up to ~35 each).
//
// Layout.  The host groups the matrices by order, largest first (a counting
// sort: `perm` lists matrix indices by position), and describes each order in
// a BatchTable: which kernel walks it, the codes per work item, the items per
// matrix, and where its items' tickets and partials start.  Items are never
// listed: a kernel decodes a ticket into (order, matrix, code chunk) from the
// table (batch_common.cuh), so a plan is O(count) to build and holds one int
// per matrix plus four doubles per item.
//
// Kernels.  Orders go to one of four persistent kernels, chosen per order by
// the tuner: one warp per item with exact fixed-point rows (k_batch here; its
// lanes share an item, so small orders need little staging), or one block per
// item with the packed double-float walk (batch_cta.cuh: 128 threads allowing
// 2 or 3 blocks per SM, or 256 threads).  Each kernel pulls tickets from its own
// counter, largest orders first.  A finalize kernel adds each matrix's item
// partials in item order (deterministic) and applies 2 (-1)^(n-1).
//
// Asynchrony.  The pointers of a call (matrix pointer array, output) are
// written into a 16-byte device argument block by a one-thread kernel just
// before the graph launch, so one cached plan (keyed by device, stream,
// orders and tuning) serves any matrices of that shape.  A new plan's buffers
// come from stream-ordered allocations on the caller's stream and its
// position list is uploaded by kernels whose parameters carry the data (no
// pinned staging, no synchronous copy), so perm_batch never waits for the
// device.  Tuning (perm_batch_autotune) is the one blocking step; untuned
// orders take built-in defaults.
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <vector>

#include "batch_common.cuh"
#include "glynn_walk.cuh"
#include "glynn_walk_fx.cuh"
#include "perm.h"
#include "perm_internal.h"

namespace perm {

constexpr int kBatchThreads = 128;
constexpr int kBatchWarps = kBatchThreads / 32;
// Per-warp shared slot (16-byte units): the FP64-row walk keeps the row-scaled
// A (n^2), w0 (n) and the row scale exponents; the fixed-point walk keeps +2A
// (n^2), v0 (n) and two int rows.
constexpr size_t kBatchSlot = (size_t)kBatchNMax * kBatchNMax + kBatchNMax + (2 * kBatchNMax * 4 + 15) / 16;
constexpr size_t kBatchSmem = kBatchSlot * kBatchWarps * 16;

template <int K, int ROWS>
__device__ __forceinline__ void batch_walk_case(int n, double2* slot, uint64_t r, uint64_t end, dd& accr, dd& acci) {
  if constexpr (K <= kBatchNMax) {
    if (n == K) {
      if constexpr (ROWS == kRowsFixed) {
        const longlong2* sP = reinterpret_cast<const longlong2*>(slot);
        const longlong2* sV0 = sP + K * K;
        const int* sEb = reinterpret_cast<const int*>(sV0 + K);
        thread_walk_c128_fx<K, kProdF64, false>(sP, nullptr, sV0, sEb, r, end, accr, acci);
      } else {
        thread_walk_c128<K, kProdF64>(slot, slot + K * K, r, end, accr, acci);
      }
      return;
    }
    batch_walk_case<K + 1, ROWS>(n, slot, r, end, accr, acci);
  }
}

// One warp per item: the warp stages its item's matrix into its own slot and
// its 32 lanes walk consecutive shares of the item's codes.
template <int ROWS>
__global__ void __launch_bounds__(kBatchThreads)
    k_batch(const BatchArgs* __restrict__ ba, const int* __restrict__ perm, const __grid_constant__ BatchTable tab,
            double* __restrict__ partials, unsigned long long* __restrict__ ticket, int* __restrict__ status) {
  extern __shared__ __align__(16) double2 bsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* slot = bsm + (size_t)warp * kBatchSlot;
  const double* const* ptrs = ba->ptrs;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    BatchItemRef item;
    if (!batch_decode(tab, kBatchWarp, perm, t, item)) break;
    const int n = item.n;
    const double2* __restrict__ A = reinterpret_cast<const double2*>(ptrs[item.matrix]);
    bool bad = false;
    // The walks multiply row values below 1 in magnitude (rows scaled by
    // powers of two); the product of the rows' scales is applied once, to the
    // item's sum, so no product chain leaves the double range however the
    // rows of A are scaled.
    int scale = 0;
    if constexpr (ROWS == kRowsFixed) {
      longlong2* sP = reinterpret_cast<longlong2*>(slot);
      longlong2* sV0 = sP + n * n;
      int* sEb = reinterpret_cast<int*>(sV0 + n);
      bad = fx_stage_warp_c128(A, n, sP, sV0, sEb, sEb + n);
      if (!bad) {
        for (int i = 0; i < n; ++i) scale += sEb[i] - 1023;
        __syncwarp();
        if (lane < n) sEb[lane] = 1023;  // products of v_i 2^-63
        __syncwarp();
      }
    } else {
      // stage row-scaled entries column-major (the single-matrix kernel's
      // layout) and w0; row i is scaled by 2^G_i, its largest part near 1
      double2* sA = slot;
      double2* sW0 = slot + n * n;
      int* sG = reinterpret_cast<int*>(sW0 + n);
      int b = 0;
      if (lane < n) {
        double mx = 0.0;
        for (int j = 0; j < n; ++j) {
          const double2 v = A[lane * n + j];
          b |= (not_finite(v.x) || not_finite(v.y)) ? 1 : 0;
          mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
        }
        sG[lane] = (mx > 0.0 && !b) ? -ilogb(mx) : 0;
      }
      bad = __any_sync(0xffffffffu, b) != 0;
      __syncwarp();
      for (int i = 0; i < n; ++i) scale -= sG[i];
      for (int idx = lane; idx < n * n; idx += 32) {
        const int i = idx / n, j = idx - i * n;
        const double2 v = A[idx];
        const int G = sG[i];
        sA[j * n + i] = make_double2(scalbn(v.x, G), scalbn(v.y, G));
      }
      __syncwarp();
      if (lane < n) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; ++j) {
          sr += sA[j * n + lane].x;
          si += sA[j * n + lane].y;
        }
        const double2 last = sA[(n - 1) * n + lane];
        sW0[lane] = make_double2(fma(-0.5, sr, last.x), fma(-0.5, si, last.y));
      }
      __syncwarp();
    }
    if (bad && lane == 0) atomicOr(status, (int)kStatusNonFinite);
    // this lane's share of the item ("distribute" over 32 lanes)
    const uint64_t q = item.count / 32, rem = item.count % 32;
    const uint64_t r = item.first + lane * q + ((uint64_t)lane < rem ? lane : rem);
    const uint64_t end = r + q + ((uint64_t)lane < rem ? 1 : 0);
    dd accr{0.0, 0.0}, acci{0.0, 0.0};
    if (!bad)
      batch_walk_case<1, ROWS>(n, slot, r, end, accr, acci);
    else
      accr = acci = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
    accr = dd_warp_sum_exact(accr, scale);  // the rows' scales applied in the exponent
    acci = dd_warp_sum_exact(acci, scale);
    if (lane == 0) {
      double* o = partials + item.partial * 4;
      o[0] = accr.hi;
      o[1] = accr.lo;
      o[2] = acci.hi;
      o[3] = acci.lo;
    }
    __syncwarp();
  }
}

// Order of the matrix at position i (orders are grouped, largest first).
__device__ __forceinline__ int order_at(const BatchTable& tab, int i) {
  for (int m = kBatchNMax; m >= 1; --m)
    if (tab.kind[m] != kBatchNone && i >= tab.mstart[m] && i < tab.mstart[m] + tab.mcount[m]) return m;
  return 0;
}

// out[2k..2k+1] = 2 (-1)^(n_k - 1) * sum of matrix k's item partials, in item
// order; one thread per position.
__global__ void k_batch_finalize(const BatchArgs* __restrict__ ba, const int* __restrict__ perm,
                                 const __grid_constant__ BatchTable tab, const double* __restrict__ partials,
                                 int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int n = order_at(tab, i);
  if (n == 0) return;
  const uint64_t ipm = tab.items_per_matrix[n];
  const uint64_t f = tab.gbase[n] + (uint64_t)(i - tab.mstart[n]) * ipm;
  dd ar{0.0, 0.0}, ai{0.0, 0.0};
  for (uint64_t t = 0; t < ipm; ++t) {
    const double* p = partials + (f + t) * 4;
    ar = dd_add(ar, dd{p[0], p[1]});
    ai = dd_add(ai, dd{p[2], p[3]});
  }
  const int k = perm[i];
  const double s = ((n - 1) & 1) ? -2.0 : 2.0;
  double* out = ba->out;
  out[2 * k] = s * __dadd_rn(ar.hi, ar.lo);
  out[2 * k + 1] = s * __dadd_rn(ai.hi, ai.lo);
}

// Device copy of a host int array, carried in the kernel's parameters (so the
// upload is stream-ordered without pinned host memory).
constexpr int kUploadInts = 4000;
struct UploadChunk {
  int v[kUploadInts];
};

__global__ void k_upload(int* __restrict__ dst, const __grid_constant__ UploadChunk c, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = c.v[i];
}

__global__ void k_set_args(BatchArgs* __restrict__ ba, const double* const* ptrs, double* out) {
  ba->ptrs = ptrs;
  ba->out = out;
}

// ---- statistics of X = |per| / sqrt(n!) per order (Secs. 3-6) ----
// stats[n * PERM_STATS_STRIDE + ...]: [0] count, [1..4] sum X^1..X^4,
// [5 + b] histogram: b = 0 for X < 1e-4, b = 1..96 for
// 10^(-4 + (b-1)/16) <= X < 10^(-4 + b/16) (16 bins per decade), b = 97 for
// X >= 100.  Two kernels: one block per chunk of kStatsChunk positions of one
// order writes the chunk's four moment sums (each thread's FP64 sums added
// exactly as 128-bit fixed-point integers over the block) and its histogram;
// then one block per order adds its chunks' records, the moments again as
// exact integer sums, the counts as integers.  Every total is independent of
// the order in which blocks and threads finish.
constexpr int kStatsEdges = 97;  // 10^(-4 + j/16), j = 0..96
constexpr int kStatsStride = 5 + kStatsEdges + 1;
constexpr int kStatsBins = kStatsEdges + 1;
constexpr int kStatsChunk = 4096;  // positions per block of the first kernel
constexpr int kStatsThreads = 256;

struct StatsParams {
  double inv_sqrt_fact[kBatchNMax + 1];
  double edges[kStatsEdges];
  int cfirst[kBatchNMax + 2];  // chunks of order m: [cfirst[m], cfirst[m + 1])
};

// Exact sums over the block of K per-thread doubles (dd.cuh: fx128); the
// totals, as double-doubles, on thread 0 (NaN if any value is non-finite).
template <int K>
__device__ __forceinline__ void block_sum_exact(const double (&v)[K], dd (&tot)[K]) {
  __shared__ int sEmax;
  __shared__ fx128 sF[K * (kStatsThreads / 32)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) sEmax = 1;
  __syncthreads();
  int e = 0;
#pragma unroll
  for (int q = 0; q < K; ++q) e = max(e, dexp_field(v[q]));
  e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
  if (lane == 0) atomicMax(&sEmax, e);
  __syncthreads();
  const int emax = sEmax;
  if (emax < 0x7FF) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const fx128 f = fx128_warp_sum(fx128_of(v[q], emax));
      if (lane == 0) sF[K * warp + q] = f;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      if (emax >= 0x7FF) {
        tot[q] = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
        continue;
      }
      fx128 f = sF[q];
      for (int w = 1; w < kStatsThreads / 32; ++w) f = fx128_add(f, sF[K * w + q]);
      tot[q] = dd_of_fx128(f, emax);
    }
  }
}

// Order of chunk c (0 if none).
__device__ __forceinline__ int stats_order_of(const StatsParams& sp, int c) {
  for (int m = 1; m <= kBatchNMax; ++m)
    if (c >= sp.cfirst[m] && c < sp.cfirst[m + 1]) return m;
  return 0;
}

// One block per chunk: moments (as double-double hi, lo pairs) to cmom[8 c ..],
// histogram to chist[kStatsBins c ..].
__global__ void __launch_bounds__(kStatsThreads)
    k_batch_stats_part(const BatchArgs* __restrict__ ba, const int* __restrict__ perm,
                       const __grid_constant__ BatchTable tab, const __grid_constant__ StatsParams sp,
                       double* __restrict__ cmom, unsigned int* __restrict__ chist) {
  __shared__ unsigned int hist[kStatsBins];
  const int c = blockIdx.x;
  const int n = stats_order_of(sp, c);
  for (int b = threadIdx.x; b < kStatsBins; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  double m[4] = {0.0, 0.0, 0.0, 0.0};
  if (n > 0) {
    const int lo_pos = tab.mstart[n] + (c - sp.cfirst[n]) * kStatsChunk;
    const int hi_pos = min(lo_pos + kStatsChunk, tab.mstart[n] + tab.mcount[n]);
    const double* out = ba->out;
    for (int i = lo_pos + (int)threadIdx.x; i < hi_pos; i += blockDim.x) {
      const int k = perm[i];
      const double re = out[2 * (size_t)k], im = out[2 * (size_t)k + 1];
      const double x = sqrt(re * re + im * im) * sp.inv_sqrt_fact[n];
      const double x2 = x * x;
      m[0] += x;
      m[1] += x2;
      m[2] += x2 * x;
      m[3] += x2 * x2;
      // bin = number of edges <= x (binary search over the ascending edges)
      int lo = 0, hi = kStatsEdges;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sp.edges[mid] <= x)
          lo = mid + 1;
        else
          hi = mid;
      }
      atomicAdd(&hist[lo], 1u);
    }
  }
  dd tot[4];
  block_sum_exact<4>(m, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      cmom[8 * (size_t)c + 2 * q] = tot[q].hi;
      cmom[8 * (size_t)c + 2 * q + 1] = tot[q].lo;
    }
  }
  for (int b = threadIdx.x; b < kStatsBins; b += blockDim.x) chist[(size_t)kStatsBins * c + b] = hist[b];
}

// One block per order: its chunks' records added (moments exactly, counts as
// integers) into stats[n * kStatsStride ..]; zeros for an order not in the batch.
__global__ void __launch_bounds__(kStatsThreads)
    k_batch_stats_final(const __grid_constant__ BatchTable tab, const __grid_constant__ StatsParams sp,
                        const double* __restrict__ cmom, const unsigned int* __restrict__ chist,
                        double* __restrict__ stats) {
  const int n = blockIdx.x;
  const int c0 = n >= 1 ? sp.cfirst[n] : 0, c1 = n >= 1 ? sp.cfirst[n + 1] : 0;
  double* st = stats + (size_t)n * kStatsStride;
  // histogram: one thread per bin, chunks in order (integer sums)
  for (int b = threadIdx.x; b < kStatsBins; b += blockDim.x) {
    unsigned long long h = 0;
    for (int c = c0; c < c1; ++c) h += chist[(size_t)kStatsBins * c + b];
    st[5 + b] = (double)h;
  }
  // moments: every thread's share of the chunks' hi and lo parts, summed exactly
  double part[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) part[q] = 0.0;
  // each thread takes at most one chunk per pass; a pass is summed exactly,
  // the passes are added in order in double-double
  dd acc[4] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
  for (int base = c0; base < c1; base += blockDim.x) {
    const int c = base + (int)threadIdx.x;
#pragma unroll
    for (int q = 0; q < 8; ++q) part[q] = c < c1 ? cmom[8 * (size_t)c + q] : 0.0;
    dd t[8];
    block_sum_exact<8>(part, t);
    if (threadIdx.x == 0)
      for (int q = 0; q < 4; ++q) acc[q] = dd_add(acc[q], dd_add(t[2 * q], t[2 * q + 1]));
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st[0] = n >= 1 && tab.kind[n] != kBatchNone ? (double)tab.mcount[n] : 0.0;
    for (int q = 0; q < 4; ++q) st[1 + q] = __dadd_rn(acc[q].hi, acc[q].lo);
  }
}

template <int ROWS>
int batch_resident_blocks_t() {
  static std::atomic<int> cached[64];  // per device; filled once, read from any host thread
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (cached[dev]) return cached[dev];
  if (cudaFuncSetAttribute(k_batch<ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<ROWS>, kBatchThreads, kBatchSmem) !=
      cudaSuccess)
    return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cached[dev] = (per_sm < 1 ? 1 : per_sm) * sms;
  return cached[dev];
}

int batch_resident_blocks_rows(RowMode rows) {
  return rows == kRowsF64 ? batch_resident_blocks_t<kRowsF64>() : batch_resident_blocks_t<kRowsFixed>();
}

int batch_resident_blocks_cta(int kind) {
  return kind == kBatchCta3 ? batch_resident_cta_minb3()
                            : kind == kBatchCta256 ? batch_resident_cta256() : batch_resident_cta_minb2();
}

cudaError_t batch_launch_warp(const BatchArgs* ba, const int* perm, const BatchTable& tab, double* partials,
                              unsigned long long* ticket, int* status, RowMode rows, cudaStream_t s) {
  const int grid = batch_resident_blocks_rows(rows);
  if (grid < 1) return cudaErrorInvalidConfiguration;
  if (rows == kRowsF64)
    k_batch<kRowsF64><<<grid, kBatchThreads, kBatchSmem, s>>>(ba, perm, tab, partials, ticket, status);
  else
    k_batch<kRowsFixed><<<grid, kBatchThreads, kBatchSmem, s>>>(ba, perm, tab, partials, ticket, status);
  return cudaGetLastError();
}

cudaError_t batch_launch_cta(int kind, const BatchArgs* ba, const int* perm, const BatchTable& tab, double* partials,
                             unsigned long long* ticket, int* status, cudaStream_t s) {
  if (kind == kBatchCta3) return batch_launch_cta_minb3(ba, perm, tab, kind, partials, ticket, status, s);
  if (kind == kBatchCta256) return batch_launch_cta256(ba, perm, tab, kind, partials, ticket, status, s);
  return batch_launch_cta_minb2(ba, perm, tab, kind, partials, ticket, status, s);
}

void preload_batch_kernels() {
  load_kernel(k_batch_finalize);
  load_kernel(k_batch_stats_part);
  load_kernel(k_batch_stats_final);
  load_kernel(k_upload);
  load_kernel(k_set_args);
  batch_resident_blocks_rows(kRowsF64);
  batch_resident_blocks_rows(kRowsFixed);
  batch_resident_cta_minb2();
  batch_resident_cta_minb3();
  batch_resident_cta256();
}

}  // namespace perm

using namespace perm;

namespace {

std::mutex g_batch_mu;
std::mutex g_stats_mu;

// ---- tuning: kernel kind and codes per thread for each (row class, device, order) ----
struct Tune {
  int L[kBatchNMax + 1] = {0};     // codes per lane (warp kernel) or per thread (block kernels); 0 = untuned
  int kind[kBatchNMax + 1] = {0};  // BatchKind; 0 = untuned
};
// row class: 0 FP64 rows, 1 exact fixed-point rows (both: warp kernel only), 2 the default arithmetic
Tune g_tune_tab[3][64];

int row_class(RowMode r) { return r == kRowsF64 ? 0 : r == kRowsFixed ? 1 : 2; }
bool warp_only(RowMode r) { return r == kRowsF64 || r == kRowsFixed; }
Tune& tune_of(int dev) { return g_tune_tab[row_class(rows_from_env())][dev]; }

// Built-in choice for an untuned order: the table perm_batch_autotune
// measured on GB300 for orders 12..28 (kind, codes per thread); below 12 the
// warp kernel, above 28 the block kernel with 2048 codes per thread.
constexpr int kTunedLo = 12, kTunedHi = 28;
constexpr int kTunedKind[kTunedHi - kTunedLo + 1] = {1, 3, 3, 3, 2, 3, 3, 3, 3, 2, 2, 2, 2, 2, 2, 2, 2};
constexpr int kTunedL[kTunedHi - kTunedLo + 1] = {64,  32,  64,  128, 128, 128,  256,  128, 128,
                                                 512, 512, 512, 512, 512, 1024, 2048, 1024};

int default_L_warp(int n) {
  // about 16 n codes per lane keeps the O(n^2) seed near 2% of the walk
  int L = 64;
  while (L < 16 * n && L < 4096) L <<= 1;
  return L;
}

void default_choice(int n, int& kind, int& L) {
  if (n >= kTunedLo && n <= kTunedHi) {
    kind = kTunedKind[n - kTunedLo];
    L = kTunedL[n - kTunedLo];
  } else if (n < kTunedLo) {
    kind = kBatchWarp;
    L = default_L_warp(n < 1 ? 1 : n);
  } else {
    kind = kBatchCta;
    L = 2048;
  }
}

struct Choice {
  int kind[kBatchNMax + 1];
  int L[kBatchNMax + 1];
};

Choice resolve_choice(int dev, RowMode rows) {
  Choice c;
  const Tune& t = g_tune_tab[row_class(rows)][dev];
  for (int n = 0; n <= kBatchNMax; ++n) {
    if (n >= 1 && t.kind[n] && t.L[n]) {
      c.kind[n] = t.kind[n];
      c.L[n] = t.L[n];
    } else if (warp_only(rows)) {
      c.kind[n] = kBatchWarp;
      c.L[n] = default_L_warp(n < 1 ? 1 : n);
    } else {
      default_choice(n, c.kind[n], c.L[n]);
    }
    if (warp_only(rows) && c.kind[n] != kBatchWarp) {
      c.kind[n] = kBatchWarp;
      c.L[n] = default_L_warp(n < 1 ? 1 : n);
    }
  }
  return c;
}

uint64_t threads_per_item(int kind) {
  return kind == kBatchWarp ? 32ull : kind == kBatchCta256 ? 256ull : (uint64_t)kBatchCtaThreads;
}

// Most work items one plan holds (2 GiB of partials).
constexpr uint64_t kMaxItems = 1ull << 26;

// Double the chunk length of the order contributing the most items until the
// batch has at most max(kMaxItems, count) items, so the partials stay bounded
// and item indices fit however large the batch.
void bound_items(const int* cnt, Choice& c, int count) {
  const uint64_t cap = std::max<uint64_t>(kMaxItems, (uint64_t)count);
  for (;;) {
    uint64_t total = 0, worst = 0;
    int wn = -1;
    for (int n = 1; n <= kBatchNMax; ++n) {
      if (!cnt[n]) continue;
      const uint64_t per_item = threads_per_item(c.kind[n]) * (uint64_t)c.L[n];
      const uint64_t each = ((1ull << (n - 1)) + per_item - 1) / per_item;
      const uint64_t t = (uint64_t)cnt[n] * each;
      total += t;
      if (each > 1 && t > worst) worst = t, wn = n;
    }
    if (total <= cap || wn < 0) break;
    c.L[wn] *= 2;
  }
}

int status_of_b(cudaError_t e) {
  if (e == cudaSuccess) return PERM_OK;
  if (e == cudaErrorMemoryAllocation) return PERM_ENOMEM;
  return PERM_ECUDA;
}

int* batch_status_word(int dev) {
  int* w = nullptr;
  return device_status_word(dev, &w) == 0 ? w : nullptr;
}

struct Plan {
  int dev = -1;
  cudaStream_t stream = nullptr;
  RowMode rows = kRowsPdf;
  std::vector<int> ns;
  Choice choice{};
  BatchTable tab{};
  int count = 0;
  void* args = nullptr;
  void* perm = nullptr;
  void* partials = nullptr;
  void* tickets = nullptr;
  cudaGraphExec_t exec = nullptr;
  Plan() = default;
  Plan(const Plan&) = delete;
  Plan& operator=(const Plan&) = delete;
  ~Plan() {
    // cudaFree waits for any launch still using the buffers (eviction and
    // perm_shutdown only)
    if (exec) cudaGraphExecDestroy(exec);
    for (void* p : {args, perm, partials, tickets})
      if (p) cudaFree(p);
  }
};

// Build a plan's layout, buffers (stream-ordered on s), uploaded position list
// and graph.  Nothing here waits for the device.
int build_plan(Plan& p, const int* ns, int count, const Choice& ch, RowMode rows, int dev, cudaStream_t s,
               int* status) {
  p.dev = dev;
  p.stream = s;
  p.rows = rows;
  p.ns.assign(ns, ns + count);
  p.choice = ch;
  p.count = count;
  int cnt[kBatchNMax + 1] = {0};
  for (int k = 0; k < count; ++k) ++cnt[ns[k]];
  // counting sort by decreasing order (stable within an order)
  int start[kBatchNMax + 1] = {0}, fill[kBatchNMax + 1] = {0};
  int pos = 0;
  for (int n = kBatchNMax; n >= 1; --n) start[n] = fill[n] = pos, pos += cnt[n];
  std::vector<int> perm(count);
  for (int k = 0; k < count; ++k) perm[fill[ns[k]]++] = k;
  BatchTable& t = p.tab;
  std::memset(&t, 0, sizeof(t));
  uint64_t kb[kBatchKinds] = {}, gb = 0;
  for (int n = kBatchNMax; n >= 1; --n) {
    if (!cnt[n]) continue;
    const int kind = ch.kind[n];
    const uint64_t per_item = threads_per_item(kind) * (uint64_t)ch.L[n];
    const uint64_t ipm = ((1ull << (n - 1)) + per_item - 1) / per_item;
    t.kind[n] = kind;
    t.mstart[n] = start[n];
    t.mcount[n] = cnt[n];
    t.per_item[n] = per_item;
    t.items_per_matrix[n] = ipm;
    t.kbase[n] = kb[kind];
    t.gbase[n] = gb;
    kb[kind] += (uint64_t)cnt[n] * ipm;
    gb += (uint64_t)cnt[n] * ipm;
  }
  for (int k = 0; k < kBatchKinds; ++k) t.kitems[k] = kb[k];
  cudaError_t e = cudaMallocAsync(&p.args, sizeof(BatchArgs), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&p.perm, (size_t)count * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&p.partials, (size_t)gb * 4 * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&p.tickets, kBatchKinds * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return status_of_b(e);
  UploadChunk chunk;
  for (int off = 0; off < count; off += kUploadInts) {
    const int len = std::min(kUploadInts, count - off);
    std::memcpy(chunk.v, perm.data() + off, (size_t)len * sizeof(int));
    k_upload<<<1, 256, 0, s>>>((int*)p.perm + off, chunk, len);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return status_of_b(e);
  // capture: ticket reset, the kernels that have items, finalize
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return status_of_b(e);
  cudaGraph_t graph = nullptr;
  int rc = PERM_OK;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const BatchArgs* ba = (const BatchArgs*)p.args;
    const int* dperm = (const int*)p.perm;
    double* parts = (double*)p.partials;
    unsigned long long* tk = (unsigned long long*)p.tickets;
    cudaError_t el = cudaMemsetAsync(tk, 0, kBatchKinds * sizeof(unsigned long long), cs);
    if (el == cudaSuccess && kb[kBatchWarp])
      el = batch_launch_warp(ba, dperm, t, parts, tk + kBatchWarp, status, rows, cs);
    if (el == cudaSuccess && kb[kBatchCta])
      el = batch_launch_cta(kBatchCta, ba, dperm, t, parts, tk + kBatchCta, status, cs);
    if (el == cudaSuccess && kb[kBatchCta3])
      el = batch_launch_cta(kBatchCta3, ba, dperm, t, parts, tk + kBatchCta3, status, cs);
    if (el == cudaSuccess && kb[kBatchCta256])
      el = batch_launch_cta(kBatchCta256, ba, dperm, t, parts, tk + kBatchCta256, status, cs);
    if (el == cudaSuccess) {
      k_batch_finalize<<<(count + 127) / 128, 128, 0, cs>>>(ba, dperm, t, parts, count);
      el = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    rc = status_of_b(el != cudaSuccess ? el : e2);
  } else {
    rc = status_of_b(e);
  }
  cudaStreamDestroy(cs);
  if (rc == PERM_OK) {
    e = cudaGraphInstantiate(&p.exec, graph, 0);
    if (e != cudaSuccess) rc = status_of_b(e);
  }
  if (graph) cudaGraphDestroy(graph);
  return rc;
}

bool same_choice(const Choice& a, const Choice& b, const int* cnt) {
  for (int n = 1; n <= kBatchNMax; ++n)
    if (cnt[n] && (a.kind[n] != b.kind[n] || a.L[n] != b.L[n])) return false;
  return true;
}

std::list<std::unique_ptr<Plan>> g_plans;  // most recent first
constexpr size_t kMaxPlans = 8;
std::atomic<int> g_plans_built{0};         // plans built by batch calls (not by tuning)

// Find or build the plan for (device, stream, row arithmetic, orders, tuning);
// the caller holds g_batch_mu.
int plan_for(const int* ns, int count, int dev, cudaStream_t s, int* status, const Choice* forced, Plan** out) {
  const RowMode rows = rows_from_env();
  int cnt[kBatchNMax + 1] = {0};
  for (int k = 0; k < count; ++k) ++cnt[ns[k]];
  Choice ch = forced ? *forced : resolve_choice(dev, rows);
  bound_items(cnt, ch, count);
  for (auto it = g_plans.begin(); it != g_plans.end(); ++it) {
    Plan* p = it->get();
    if (p->dev == dev && p->stream == s && p->rows == rows && p->count == count &&
        std::memcmp(p->ns.data(), ns, (size_t)count * sizeof(int)) == 0 && same_choice(p->choice, ch, cnt)) {
      g_plans.splice(g_plans.begin(), g_plans, it);
      *out = p;
      return PERM_OK;
    }
  }
  auto np = std::make_unique<Plan>();
  int rc = build_plan(*np, ns, count, ch, rows, dev, s, status);
  if (rc) return rc;
  ++g_plans_built;
  g_plans.push_front(std::move(np));
  while (g_plans.size() > kMaxPlans) g_plans.pop_back();
  *out = g_plans.front().get();
  return PERM_OK;
}

int launch_plan(Plan* p, const double* const* ptrs, double* out, cudaStream_t s) {
  k_set_args<<<1, 1, 0, s>>>((BatchArgs*)p->args, ptrs, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return status_of_b(e);
  return status_of_b(cudaGraphLaunch(p->exec, s));
}

// ---- tuning (blocking; perm_batch_autotune only) ----
// Time one (kind, L) for order n on a synthetic batch of m copies of one
// matrix; returns the best of two timed launches after a warm-up.
int time_choice(int n, int kind, int L, int m, const double* const* d_ptrs, double* d_out, int dev, int* status,
                cudaStream_t s, double* ms_out) {
  std::vector<int> ns(m, n);
  Choice ch = resolve_choice(dev, rows_from_env());
  ch.kind[n] = kind;
  ch.L[n] = L;
  Plan p;
  int rc = build_plan(p, ns.data(), m, ch, rows_from_env(), dev, s, status);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3 && rc == PERM_OK; ++rep) {
    cudaEventRecord(e0, s);
    rc = launch_plan(&p, d_ptrs, d_out, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = PERM_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = best;
  return rc;
}

int autotune_order(int dev, int n) {
  const RowMode rows = rows_from_env();
  // synthetic matrix (fixed linear congruential values in [-1, 1)), replicated
  // so the batch carries at least 2^24 codes
  std::vector<double> h(2 * n * n);
  uint64_t st = 0x9E3779B97F4A7C15ull ^ (uint64_t)n;
  for (auto& v : h) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    v = (double)(int64_t)(st >> 11) / (double)(1ull << 52) - 1.0;
  }
  const uint64_t per = 1ull << (n - 1);
  const int m = (int)std::max<uint64_t>(1, (1ull << 24) / per);
  int* status = batch_status_word(dev);
  if (!status) return PERM_ENOMEM;
  void *dA = nullptr, *dptrs = nullptr, *dout = nullptr;
  cudaStream_t s = nullptr;
  int rc = PERM_OK;
  if (cudaMalloc(&dA, h.size() * sizeof(double)) != cudaSuccess || cudaMalloc(&dptrs, (size_t)m * sizeof(double*)) != cudaSuccess ||
      cudaMalloc(&dout, (size_t)m * 2 * sizeof(double)) != cudaSuccess)
    rc = PERM_ENOMEM;
  if (rc == PERM_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) rc = PERM_ECUDA;
  if (rc == PERM_OK) {
    cudaMemcpy(dA, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
    std::vector<const double*> hp(m, (const double*)dA);
    cudaMemcpy(dptrs, hp.data(), (size_t)m * sizeof(double*), cudaMemcpyHostToDevice);
  }
  double best_rate = 0.0;
  int best_kind = kBatchWarp, best_L = default_L_warp(n);
  if (!warp_only(rows)) default_choice(n, best_kind, best_L);
  const int kinds[4] = {kBatchWarp, kBatchCta, kBatchCta3, kBatchCta256};
  for (int ki = 0; ki < 4 && rc == PERM_OK; ++ki) {
    const int kind = kinds[ki];
    if (kind != kBatchWarp && warp_only(rows)) continue;
    for (int L = 16; L <= 8192 && rc == PERM_OK; L <<= 1) {
      if (threads_per_item(kind) * (uint64_t)L > per * 4 && L > 16) break;  // items far larger than a matrix
      double ms = 0;
      rc = time_choice(n, kind, L, m, (const double* const*)dptrs, (double*)dout, dev, status, s, &ms);
      if (rc) break;
      const double rate = (double)per * m / ms;
      if (rate > best_rate * 1.01) best_rate = rate, best_kind = kind, best_L = L;
    }
  }
  if (s) cudaStreamDestroy(s);
  for (void* p : {dA, dptrs, dout})
    if (p) cudaFree(p);
  if (rc) return rc;
  tune_of(dev).kind[n] = best_kind;
  tune_of(dev).L[n] = best_L;
  return PERM_OK;
}

}  // namespace

extern "C" {

int perm_batch_tuning(int device, int* L, int* kind, int set) {
  if (!L || !kind) return PERM_ENULL;
  if (device < 0 || device >= 64) return PERM_EINVAL;
  if (set) {
    // every entry 0 (untuned) or a power of two in 16 .. 2^24 codes, with a kind 1..4
    for (int n = 1; n <= kBatchNMax; ++n) {
      const int v = L[n], k = kind[n];
      if ((v == 0) != (k == 0)) return PERM_EINVAL;
      if (v != 0 && (v < 16 || v > (1 << 24) || (v & (v - 1)) != 0)) return PERM_EINVAL;
      if (k < 0 || k >= kBatchKinds) return PERM_EINVAL;
    }
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  Tune& t = g_tune_tab[row_class(rows_from_env())][device];
  for (int n = 0; n <= kBatchNMax; ++n) {
    if (set) {
      t.L[n] = n == 0 ? 0 : L[n];
      t.kind[n] = n == 0 ? 0 : kind[n];
    } else {
      L[n] = t.L[n];
      kind[n] = t.kind[n];
    }
  }
  return PERM_OK;
}

int perm_batch_autotune(int n_lo, int n_hi) {
  TraceRange trace("perm_batch_autotune");
  if (n_lo < 1 || n_hi > kBatchNMax || n_lo > n_hi) return PERM_EINVAL;
  int count = 0, dev = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return PERM_ECUDA;
  ensure_kernels_loaded();
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (int n = n_lo; n <= n_hi; ++n) {
    int rc = autotune_order(dev, n);
    if (rc) return rc;
  }
  return PERM_OK;
}

static int batch_run(const double* const* ptrs, const int* ns, int count, double* out, void* stream, double* stats) {
  if (!ptrs || !ns || !out) return PERM_ENULL;
  if (count < 1) return PERM_EINVAL;
  for (int k = 0; k < count; ++k)
    if (ns[k] < 1 || ns[k] > kBatchNMax) return PERM_EINVAL;
  int ndev = 0, dev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return PERM_ECUDA;
  ensure_kernels_loaded();
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  int* status = batch_status_word(dev);
  if (!status) return PERM_ENOMEM;
  Plan* plan = nullptr;
  int rc = plan_for(ns, count, dev, s, status, nullptr, &plan);
  if (rc) return rc;
  rc = launch_plan(plan, ptrs, out, s);
  if (rc || !stats) return rc;
  StatsParams sp;
  for (int n = 0; n <= kBatchNMax; ++n) {
    double f = 1.0;
    for (int t = 2; t <= n; ++t) f *= (double)t;
    sp.inv_sqrt_fact[n] = 1.0 / std::sqrt(f);
  }
  for (int j = 0; j < kStatsEdges; ++j) sp.edges[j] = std::pow(10.0, -4.0 + (double)j / 16.0);
  sp.cfirst[0] = sp.cfirst[1] = 0;
  for (int m = 1; m <= kBatchNMax; ++m) {
    const int c = plan->tab.kind[m] != kBatchNone ? (plan->tab.mcount[m] + kStatsChunk - 1) / kStatsChunk : 0;
    sp.cfirst[m + 1] = sp.cfirst[m] + c;
  }
  const int nchunks = sp.cfirst[kBatchNMax + 1];
  if (nchunks < 1) return PERM_EINVAL;
  const size_t mom_bytes = (size_t)nchunks * 8 * sizeof(double);
  char* scratch = nullptr;
  if (cudaMallocAsync((void**)&scratch, mom_bytes + (size_t)nchunks * kStatsBins * sizeof(unsigned int), s) !=
      cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  double* cmom = reinterpret_cast<double*>(scratch);
  unsigned int* chist = reinterpret_cast<unsigned int*>(scratch + mom_bytes);
  k_batch_stats_part<<<nchunks, kStatsThreads, 0, s>>>((const BatchArgs*)plan->args, (const int*)plan->perm,
                                                       plan->tab, sp, cmom, chist);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_batch_stats_final<<<kBatchNMax + 1, kStatsThreads, 0, s>>>(plan->tab, sp, cmom, chist, stats);
    e = cudaGetLastError();
  }
  cudaFreeAsync(scratch, s);
  return status_of_b(e);
}

int perm_batch_plans(int* built) {
  if (!built) return PERM_ENULL;
  *built = g_plans_built.load();
  return PERM_OK;
}

int perm_batch(const double* const* ptrs, const int* ns, int count, double* out, void* stream) {
  TraceRange trace("perm_batch");
  return batch_run(ptrs, ns, count, out, stream, nullptr);
}

int perm_batch_stats(const double* const* ptrs, const int* ns, int count, double* out, double* stats, void* stream) {
  TraceRange trace("perm_batch_stats");
  if (!stats) return PERM_ENULL;
  std::lock_guard<std::mutex> lk(g_stats_mu);
  return batch_run(ptrs, ns, count, out, stream, stats);
}

}  // extern "C"

namespace perm {

void batch_release_plans() {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  g_plans.clear();
}

}  // namespace perm

// Batched permanents: many independent complex matrices of uneven order in
// one persistent launch (the random-matrix studies of Secs. 3-6 compute
// 10^5..10^7 permanents of orders up to ~35 each).
//
// Work is cut into (matrix, code range) items of 32 lanes x L codes, L tuned
// per order; the host sorts items by decreasing order (largest work first)
// and each warp of the persistent grid pulls the next item from an atomic
// ticket, stages that matrix into its own shared-memory slot, walks its range
// with the same per-thread Gray walk as the single-matrix kernel, and writes
// a double-double partial per item.  A second kernel adds each matrix's item
// partials in item order (deterministic) and applies 2 (-1)^(n-1).  The pair
// of launches (plus the ticket reset) is captured once per (device, stream,
// pointers, orders) into a CUDA graph and replayed.
//
// Tuning: for each order n the codes-per-lane L is chosen by timing the
// candidates on a synthetic batch the first time n is seen (or by
// perm_batch_autotune); PERM_BATCH_TUNE=0 keeps the built-in default.
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

#include "glynn_walk.cuh"
#include "glynn_walk_fx.cuh"
#include "perm.h"
#include "perm_internal.h"

namespace perm {

constexpr int kBatchNMax = 32;
constexpr int kBatchThreads = 128;
constexpr int kBatchWarps = kBatchThreads / 32;
// Per-warp shared slot (16-byte units): the FP64-row walk keeps A (n^2) and
// w0 (n); the fixed-point walk keeps +2A (n^2), v0 (n) and two int rows.
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

template <int ROWS>
__global__ void __launch_bounds__(kBatchThreads) k_batch(const double* const* __restrict__ ptrs,
                                                         const BatchItem* __restrict__ items, int nitems,
                                                         double* __restrict__ item_partials,
                                                         unsigned int* __restrict__ ticket, int* __restrict__ status) {
  extern __shared__ __align__(16) double2 bsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* slot = bsm + (size_t)warp * kBatchSlot;
  for (;;) {
    unsigned int it = 0;
    if (lane == 0) it = atomicAdd(ticket, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned int)nitems) break;
    const BatchItem item = items[it];
    const int n = (int)item.n;
    const double2* __restrict__ A = reinterpret_cast<const double2*>(ptrs[item.matrix]);
    bool bad = false;
    if constexpr (ROWS == kRowsFixed) {
      longlong2* sP = reinterpret_cast<longlong2*>(slot);
      longlong2* sV0 = sP + n * n;
      int* sEb = reinterpret_cast<int*>(sV0 + n);
      bad = fx_stage_warp_c128(A, n, sP, sV0, sEb, sEb + n);
    } else {
      // stage column-major (the single-matrix kernel's layout) and w0
      double2* sA = slot;
      double2* sW0 = slot + n * n;
      int b = 0;
      for (int idx = lane; idx < n * n; idx += 32) {
        const int i = idx / n, j = idx - i * n;
        const double2 v = A[idx];
        b |= (not_finite(v.x) || not_finite(v.y)) ? 1 : 0;
        sA[j * n + i] = v;
      }
      bad = __any_sync(0xffffffffu, b) != 0;
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
    accr = dd_warp_sum(accr);
    acci = dd_warp_sum(acci);
    if (lane == 0) {
      double* o = item_partials + (size_t)it * 4;
      o[0] = accr.hi;
      o[1] = accr.lo;
      o[2] = acci.hi;
      o[3] = acci.lo;
    }
    __syncwarp();
  }
}

// out[2k..2k+1] = 2 (-1)^(n_k - 1) * sum of matrix k's item partials, in item order.
__global__ void k_batch_finalize(const double* __restrict__ item_partials, const int* __restrict__ mat_first,
                                 const int* __restrict__ mat_items, const int* __restrict__ mat_n, int count,
                                 double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  dd ar{0.0, 0.0}, ai{0.0, 0.0};
  const int f = mat_first[k], c = mat_items[k];
  for (int t = 0; t < c; ++t) {
    const double* p = item_partials + (size_t)(f + t) * 4;
    ar = dd_add(ar, dd{p[0], p[1]});
    ai = dd_add(ai, dd{p[2], p[3]});
  }
  const double s = ((mat_n[k] - 1) & 1) ? -2.0 : 2.0;
  out[2 * k] = s * __dadd_rn(ar.hi, ar.lo);
  out[2 * k + 1] = s * __dadd_rn(ai.hi, ai.lo);
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

int batch_resident_blocks() { return batch_resident_blocks_rows(rows_from_env()); }

// ---- statistics of X = |per| / sqrt(n!) per order (Secs. 3-6) ----
// stats[n * PERM_STATS_STRIDE + ...]: [0] count, [1..4] sum X^1..X^4,
// [5 + b] histogram: b = 0 for X < 1e-4, b = 1..96 for
// 10^(-4 + (b-1)/16) <= X < 10^(-4 + b/16) (16 bins per decade), b = 97 for
// X >= 100.  One block per order; every sum is formed in a fixed order
// (double-double per thread, fixed tree), counts are integer atomics.
constexpr int kStatsEdges = 97;  // 10^(-4 + j/16), j = 0..96
constexpr int kStatsStride = 5 + kStatsEdges + 1;

struct StatsParams {
  double inv_sqrt_fact[kBatchNMax + 1];
  double edges[kStatsEdges];
};

__global__ void __launch_bounds__(256) k_batch_stats(const double* __restrict__ out, const int* __restrict__ ns,
                                                     int count, StatsParams sp, double* __restrict__ stats) {
  const int n = blockIdx.x;
  __shared__ unsigned int hist[kStatsEdges + 1];
  __shared__ unsigned int cnt;
  __shared__ dd red[4 * 8];
  for (int b = threadIdx.x; b <= kStatsEdges; b += blockDim.x) hist[b] = 0;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  dd m1{0, 0}, m2{0, 0}, m3{0, 0}, m4{0, 0};
  unsigned int c = 0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) {
    if (ns[k] != n) continue;
    const double re = out[2 * (size_t)k], im = out[2 * (size_t)k + 1];
    const double x = sqrt(re * re + im * im) * sp.inv_sqrt_fact[n];
    const double x2 = x * x;
    m1 = dd_add_d(m1, x);
    m2 = dd_add_d(m2, x2);
    m3 = dd_add_d(m3, x2 * x);
    m4 = dd_add_d(m4, x2 * x2);
    ++c;
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
  m1 = dd_warp_sum(m1);
  m2 = dd_warp_sum(m2);
  m3 = dd_warp_sum(m3);
  m4 = dd_warp_sum(m4);
  for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[4 * warp] = m1;
    red[4 * warp + 1] = m2;
    red[4 * warp + 2] = m3;
    red[4 * warp + 3] = m4;
    atomicAdd(&cnt, c);
  }
  __syncthreads();
  double* st = stats + (size_t)n * kStatsStride;
  if (threadIdx.x == 0) {
    dd t[4] = {red[0], red[1], red[2], red[3]};
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      for (int q = 0; q < 4; ++q) t[q] = dd_add(t[q], red[4 * w + q]);
    st[0] = (double)cnt;
    for (int q = 0; q < 4; ++q) st[1 + q] = __dadd_rn(t[q].hi, t[q].lo);
  }
  for (int b = threadIdx.x; b <= kStatsEdges; b += blockDim.x) st[5 + b] = (double)hist[b];
}

void preload_batch_kernels() {
  load_kernel(k_batch_finalize);
  load_kernel(k_batch_stats);
}

}  // namespace perm

using namespace perm;

namespace {

std::mutex g_batch_mu;
std::mutex g_stats_mu;

// ---- tuning table: codes per lane L for each (device, order) ----
struct Tune {
  int L[kBatchNMax + 1] = {0};
};
Tune g_tune_tab[2][64];  // [row mode][device]

// Tuning table of the row arithmetic currently selected (PERM_ROWS).
Tune& tune_of(int dev) { return g_tune_tab[rows_from_env() == kRowsF64 ? 0 : 1][dev]; }

int default_L(int n) {
  // about 16 n codes per lane keeps the O(n^2) seed near 2% of the walk
  int L = 64;
  while (L < 16 * n && L < 4096) L <<= 1;
  return L;
}

bool tuning_enabled() {
  const char* e = std::getenv("PERM_BATCH_TUNE");
  return !(e && e[0] == '0');
}

int status_of_b(cudaError_t e) {
  if (e == cudaSuccess) return PERM_OK;
  if (e == cudaErrorMemoryAllocation) return PERM_ENOMEM;
  return PERM_ECUDA;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

int* batch_status_word(int dev) {
  int* w = nullptr;
  return device_status_word(dev, &w) == 0 ? w : nullptr;
}

// Build the item list for `ns` with the given per-order L; matrices sorted
// by decreasing order, each matrix's items contiguous.
void build_items(const int* ns, int count, const int* Ltab, std::vector<BatchItem>& items, std::vector<int>& mfirst,
                 std::vector<int>& mcount) {
  std::vector<int> order(count);
  for (int k = 0; k < count; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ns[a] > ns[b]; });
  items.clear();
  mfirst.assign(count, 0);
  mcount.assign(count, 0);
  for (int k : order) {
    const int n = ns[k];
    const uint64_t total = 1ull << (n - 1);
    const uint64_t per_item = 32ull * (uint64_t)Ltab[n];
    mfirst[k] = (int)items.size();
    for (uint64_t f = 0; f < total; f += per_item) {
      BatchItem it;
      it.matrix = (uint32_t)k;
      it.n = (uint32_t)n;
      it.first = f;
      it.count = std::min(per_item, total - f);
      items.push_back(it);
    }
    mcount[k] = (int)items.size() - mfirst[k];
  }
}

// Most work items one plan holds (1.5 GiB of item list, 2 GiB of partials).
constexpr uint64_t kMaxItems = 1ull << 26;

// Chunk lengths for one batch: the tuned lengths, doubled for the order that
// contributes the most items until the batch has at most
// max(kMaxItems, count) items, so the item list and its partials stay bounded
// and item indices fit in an int however large the batch.
void plan_lengths(const int* ns, int count, const int* Ltune, int* Leff) {
  uint64_t cnt[kBatchNMax + 1] = {0};
  for (int k = 0; k < count; ++k) ++cnt[ns[k]];
  for (int n = 0; n <= kBatchNMax; ++n) Leff[n] = Ltune[n] ? Ltune[n] : default_L(n < 1 ? 1 : n);
  const uint64_t cap = std::max<uint64_t>(kMaxItems, (uint64_t)count);
  for (;;) {
    uint64_t total = 0, worst = 0;
    int wn = -1;
    for (int n = 1; n <= kBatchNMax; ++n) {
      if (!cnt[n]) continue;
      const uint64_t per_item = 32ull * (uint64_t)Leff[n];
      const uint64_t each = ((1ull << (n - 1)) + per_item - 1) / per_item;
      const uint64_t t = cnt[n] * each;
      total += t;
      if (each > 1 && t > worst) worst = t, wn = n;
    }
    if (total <= cap || wn < 0) break;
    Leff[wn] *= 2;
  }
}

struct Plan {
  int dev = -1;
  cudaStream_t stream = nullptr;
  const void* ptrs = nullptr;
  void* out = nullptr;
  std::vector<int> ns;
  std::vector<int> Ls;
  RowMode rows = kRowsFixed;
  DevBuf items, partials, mfirst, mcount, mn, ticket;
  int nitems = 0;
  cudaGraphExec_t exec = nullptr;
  ~Plan() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

std::list<std::unique_ptr<Plan>> g_plans;  // most recent first
constexpr size_t kMaxPlans = 8;

int enqueue_batch(const double* const* ptrs, const BatchItem* d_items, int nitems, double* d_partials,
                  const int* d_mfirst, const int* d_mcount, const int* d_mn, int count, unsigned int* d_ticket,
                  double* out, int* status, cudaStream_t s, RowMode rows) {
  const int grid = batch_resident_blocks_rows(rows);
  if (grid < 1) return PERM_ECUDA;
  cudaError_t e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return status_of_b(e);
  if (rows != kRowsF64)
    k_batch<kRowsFixed><<<grid, kBatchThreads, kBatchSmem, s>>>(ptrs, d_items, nitems, d_partials, d_ticket, status);
  else
    k_batch<kRowsF64><<<grid, kBatchThreads, kBatchSmem, s>>>(ptrs, d_items, nitems, d_partials, d_ticket, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return status_of_b(e);
  if (out) {
    k_batch_finalize<<<(count + 127) / 128, 128, 0, s>>>(d_partials, d_mfirst, d_mcount, d_mn, count, out);
    e = cudaGetLastError();
  }
  return status_of_b(e);
}

// Time one candidate L for order n on a synthetic batch (blocking).
int time_candidate(int n, int L, const double* const* d_ptrs, int m, double* ms_out) {
  std::vector<int> ns(m, n);
  int Ltab[kBatchNMax + 1];
  for (int k = 0; k <= kBatchNMax; ++k) Ltab[k] = L;
  std::vector<BatchItem> items;
  std::vector<int> mf, mc;
  build_items(ns.data(), m, Ltab, items, mf, mc);
  DevBuf di, dp, dt;
  if (cudaMalloc(&di.p, items.size() * sizeof(BatchItem)) != cudaSuccess) return PERM_ENOMEM;
  if (cudaMalloc(&dp.p, items.size() * 4 * sizeof(double)) != cudaSuccess) return PERM_ENOMEM;
  if (cudaMalloc(&dt.p, sizeof(unsigned int)) != cudaSuccess) return PERM_ENOMEM;
  cudaMemcpy(di.p, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
  int dev = 0;
  cudaGetDevice(&dev);
  int* status = batch_status_word(dev);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int rc = PERM_OK;
  for (int rep = 0; rep < 3 && rc == PERM_OK; ++rep) {
    cudaEventRecord(e0, nullptr);
    rc = enqueue_batch(d_ptrs, (BatchItem*)di.p, (int)items.size(), (double*)dp.p, nullptr, nullptr, nullptr, 0,
                       (unsigned int*)dt.p, nullptr, status, nullptr, rows_from_env());
    cudaEventRecord(e1, nullptr);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = PERM_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = best;
  return rc;
}

int autotune_order(int dev, int n) {
  if (tune_of(dev).L[n]) return PERM_OK;
  if (!tuning_enabled() || n < 4) {
    tune_of(dev).L[n] = default_L(n);
    return PERM_OK;
  }
  // synthetic matrix (fixed linear congruential values in [-1, 1)), replicated
  // so the batch carries at least 2^24 codes
  std::vector<double> h(2 * n * n);
  uint64_t st = 0x9E3779B97F4A7C15ull ^ (uint64_t)n;
  for (auto& v : h) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    v = (double)(int64_t)(st >> 11) / (double)(1ull << 52) - 1.0;
  }
  const uint64_t per = 1ull << (n - 1);
  int m = (int)std::max<uint64_t>(1, (1ull << 24) / per);
  DevBuf dA, dptrs;
  if (cudaMalloc(&dA.p, h.size() * sizeof(double)) != cudaSuccess) return PERM_ENOMEM;
  if (cudaMalloc(&dptrs.p, (size_t)m * sizeof(double*)) != cudaSuccess) return PERM_ENOMEM;
  cudaMemcpy(dA.p, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
  std::vector<const double*> hp(m, (const double*)dA.p);
  cudaMemcpy(dptrs.p, hp.data(), (size_t)m * sizeof(double*), cudaMemcpyHostToDevice);
  double best_rate = 0.0;
  int bestL = default_L(n);
  for (int L = 16; L <= 8192; L <<= 1) {
    if (32ull * L > per * 4 && L > 16) break;  // items much larger than a matrix: no new candidates
    double ms = 0;
    int rc = time_candidate(n, L, (const double* const*)dptrs.p, m, &ms);
    if (rc) return rc;
    const double rate = (double)per * m / ms;
    if (rate > best_rate * 1.01) best_rate = rate, bestL = L;
  }
  tune_of(dev).L[n] = bestL;
  return PERM_OK;
}

}  // namespace

extern "C" {

int perm_batch_tuning(int device, int* L, int set) {
  if (!L) return PERM_ENULL;
  if (device < 0 || device >= 64) return PERM_EINVAL;
  if (set) {
    // every entry 0 (not tuned) or a power of two in 16 .. 2^24 codes per lane
    for (int n = 0; n <= kBatchNMax; ++n) {
      const int v = L[n];
      if (v != 0 && (v < 16 || v > (1 << 24) || (v & (v - 1)) != 0)) return PERM_EINVAL;
    }
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  Tune& t = g_tune_tab[rows_from_env() == kRowsF64 ? 0 : 1][device];
  for (int n = 0; n <= kBatchNMax; ++n) {
    if (set)
      t.L[n] = n == 0 ? 0 : L[n];
    else
      L[n] = t.L[n];
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
    tune_of(dev).L[n] = 0;
    int rc = autotune_order(dev, n);
    if (rc) return rc;
  }
  return PERM_OK;
}

static int batch_run(const double* const* ptrs, const int* ns, int count, double* out, void* stream,
                     const int** dev_ns) {
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
  if (batch_resident_blocks() < 1) return PERM_ECUDA;

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  bool seen[kBatchNMax + 1] = {false};
  for (int k = 0; k < count; ++k) seen[ns[k]] = true;
  for (int n = 1; n <= kBatchNMax; ++n) {
    if (!seen[n] || tune_of(dev).L[n]) continue;
    if (cap != cudaStreamCaptureStatusNone) {
      tune_of(dev).L[n] = default_L(n);  // no timing while the caller captures
    } else {
      int rc = autotune_order(dev, n);
      if (rc) return rc;
    }
  }

  // plan lookup
  Plan* plan = nullptr;
  for (auto it = g_plans.begin(); it != g_plans.end(); ++it) {
    Plan* p = it->get();
    if (p->dev == dev && p->stream == s && p->ptrs == (const void*)ptrs && p->out == (void*)out &&
        p->rows == rows_from_env() &&
        (int)p->ns.size() == count && std::memcmp(p->ns.data(), ns, count * sizeof(int)) == 0) {
      bool sameL = true;
      for (int n = 1; n <= kBatchNMax; ++n)
        if (seen[n] && p->Ls[n] != tune_of(dev).L[n]) sameL = false;
      if (!sameL) break;
      g_plans.splice(g_plans.begin(), g_plans, it);
      plan = p;
      break;
    }
  }
  if (!plan) {
    auto np = std::make_unique<Plan>();
    np->dev = dev;
    np->stream = s;
    np->ptrs = ptrs;
    np->out = out;
    np->ns.assign(ns, ns + count);
    np->rows = rows_from_env();
    np->Ls.assign(tune_of(dev).L, tune_of(dev).L + kBatchNMax + 1);
    std::vector<BatchItem> items;
    std::vector<int> mf, mc;
    int Leff[kBatchNMax + 1];
    plan_lengths(ns, count, tune_of(dev).L, Leff);
    build_items(ns, count, Leff, items, mf, mc);
    if (items.size() > (size_t)std::max<uint64_t>(kMaxItems, (uint64_t)count)) return PERM_ENOMEM;
    np->nitems = (int)items.size();
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&np->items.p, items.size() * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMalloc(&np->partials.p, items.size() * 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&np->mfirst.p, count * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&np->mcount.p, count * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&np->mn.p, count * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&np->ticket.p, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpy(np->items.p, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(np->mfirst.p, mf.data(), count * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(np->mcount.p, mc.data(), count * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(np->mn.p, ns, count * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return status_of_b(e);
    // capture ticket reset + persistent kernel + finalize into a graph
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return status_of_b(e);
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = PERM_OK;
    if (e == cudaSuccess) {
      rc = enqueue_batch(ptrs, (BatchItem*)np->items.p, np->nitems, (double*)np->partials.p, (int*)np->mfirst.p,
                         (int*)np->mcount.p, (int*)np->mn.p, count, (unsigned int*)np->ticket.p, out, status, cs,
                         np->rows);
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (rc == PERM_OK && e2 != cudaSuccess) rc = status_of_b(e2);
    } else {
      rc = status_of_b(e);
    }
    cudaStreamDestroy(cs);
    if (rc == PERM_OK) {
      e = cudaGraphInstantiate(&np->exec, graph, 0);
      if (e != cudaSuccess) rc = status_of_b(e);
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc) return rc;
    g_plans.push_front(std::move(np));
    while (g_plans.size() > kMaxPlans) g_plans.pop_back();
    plan = g_plans.front().get();
  }
  if (dev_ns) *dev_ns = (const int*)plan->mn.p;
  return status_of_b(cudaGraphLaunch(plan->exec, s));
}

int perm_batch(const double* const* ptrs, const int* ns, int count, double* out, void* stream) {
  TraceRange trace("perm_batch");
  return batch_run(ptrs, ns, count, out, stream, nullptr);
}

int perm_batch_stats(const double* const* ptrs, const int* ns, int count, double* out, double* stats, void* stream) {
  TraceRange trace("perm_batch_stats");
  if (!stats) return PERM_ENULL;
  const int* d_ns = nullptr;
  std::lock_guard<std::mutex> lk(g_stats_mu);
  int rc = batch_run(ptrs, ns, count, out, stream, &d_ns);
  if (rc) return rc;
  StatsParams sp;
  for (int n = 0; n <= kBatchNMax; ++n) {
    double f = 1.0;
    for (int t = 2; t <= n; ++t) f *= (double)t;
    sp.inv_sqrt_fact[n] = 1.0 / std::sqrt(f);
  }
  for (int j = 0; j < kStatsEdges; ++j) sp.edges[j] = std::pow(10.0, -4.0 + (double)j / 16.0);
  k_batch_stats<<<kBatchNMax + 1, 256, 0, (cudaStream_t)stream>>>(out, d_ns, count, sp, stats);
  return status_of_b(cudaGetLastError());
}

}  // extern "C"

namespace perm {

void batch_release_plans() {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  g_plans.clear();
}

}  // namespace perm

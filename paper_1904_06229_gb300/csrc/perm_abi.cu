// C ABI of libperm.so (declarations and contracts in include/perm.h).
//
// Host side only marshals: validates arguments, stages host buffers through
// stream-ordered scratch, splits long code ranges into bounded launches, and
// enqueues the kernels.  Every arithmetic step of the permanent runs in the
// CUDA kernels of this library.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>

#include <nvtx3/nvToolsExt.h>

#include "dd.cuh"
#include "perm.h"
#include "perm_internal.h"

namespace perm {

// ---- reduction of per-block dd partials (App. A "permanent":
// S = 2 (-1)^n sum_k S_k with the partials kept in an array, Sec. 2.B) ----
// The partials are added exactly as 128-bit fixed-point integers (dd.cuh:
// fx128), so the total does not depend on the order of the blocks and the
// FP64 pipe converts only the one result.  At most kFinMaxParts partials
// (2 doubles each per component: within the 2^13-value headroom).
constexpr int kFinThreads = 256;
constexpr int kFinMaxParts = 4096;

__global__ void __launch_bounds__(kFinThreads) k_finalize(const double* __restrict__ partials, int nparts, int cplx,
                                                          int n, int mode, double* __restrict__ out) {
  __shared__ fx128 sF[2 * (kFinThreads / 32)];
  __shared__ int sEmax;
  const int stride = cplx ? 4 : 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) sEmax = 1;
  __syncthreads();
  int e = 0;
  for (int k = threadIdx.x; k < nparts; k += kFinThreads) {
    const double* p = partials + (size_t)k * stride;
    for (int q = 0; q < stride; ++q) e = max(e, dexp_field(p[q]));
  }
  e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
  if (lane == 0) atomicMax(&sEmax, e);
  __syncthreads();
  const int emax = sEmax;
  if (emax < 0x7FF) {
    fx128 fr{0, 0}, fi{0, 0};
    for (int k = threadIdx.x; k < nparts; k += kFinThreads) {
      const double* p = partials + (size_t)k * stride;
      fr = fx128_add(fr, fx128_add(fx128_of(p[0], emax), fx128_of(p[1], emax)));
      if (cplx) fi = fx128_add(fi, fx128_add(fx128_of(p[2], emax), fx128_of(p[3], emax)));
    }
    fr = fx128_warp_sum(fr);
    fi = fx128_warp_sum(fi);
    if (lane == 0) {
      sF[2 * warp] = fr;
      sF[2 * warp + 1] = fi;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    dd tr, ti;
    if (emax >= 0x7FF) {
      tr = ti = dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
    } else {
      fx128 fr = sF[0], fi = sF[1];
      for (int w = 1; w < kFinThreads / 32; ++w) {
        fr = fx128_add(fr, sF[2 * w]);
        fi = fx128_add(fi, sF[2 * w + 1]);
      }
      tr = dd_of_fx128(fr, emax);
      ti = dd_of_fx128(fi, emax);
    }
    if (mode == 0 || mode == 2 || mode == 3) {
      // mode 0: per = 2 (-1)^(n-1) * sum (halved Glynn form)
      // mode 2: per = (-1)^n * sum (Ryser's un-halved form)
      // mode 3: per = 2^(1-n) * sum (Glynn's form with column multiplicities)
      const double s = mode == 0 ? (((n - 1) & 1) ? -2.0 : 2.0)
                       : mode == 2 ? ((n & 1) ? -1.0 : 1.0)
                                   : __hiloint2double((1023 + 1 - n) << 20, 0);  // exact power of two
      out[0] = s * __dadd_rn(tr.hi, tr.lo);
      if (cplx) out[1] = s * __dadd_rn(ti.hi, ti.lo);
    } else {
      out[0] = tr.hi;
      out[1] = tr.lo;
      if (cplx) {
        out[2] = ti.hi;
        out[3] = ti.lo;
      }
    }
  }
}

void preload_abi_kernels() { load_kernel(k_finalize); }

cudaError_t finalize_launch(const double* partials, int nparts, bool cplx, int n, int mode, double* out,
                            cudaStream_t stream) {
  if (nparts < 1 || nparts > kFinMaxParts) return cudaErrorInvalidValue;
  k_finalize<<<1, kFinThreads, 0, stream>>>(partials, nparts, cplx ? 1 : 0, n, mode, out);
  return cudaGetLastError();
}

namespace {
std::mutex g_status_mu;
int* g_status_words[64] = {nullptr};
}  // namespace

int device_status_word(int dev, int** out) {
  int** words = g_status_words;
  if (dev < 0 || dev >= 64) return -3;
  std::lock_guard<std::mutex> lk(g_status_mu);
  if (!words[dev]) {
    int* p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(int));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? -6 : -3;
    e = cudaMemset(p, 0, sizeof(int));
    if (e != cudaSuccess) {
      cudaFree(p);
      return -3;
    }
    words[dev] = p;
  }
  *out = words[dev];
  return 0;
}

TraceRange::TraceRange(const char* name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }

bool fault_injected(const char* stage) {
  static std::mutex mu;
  static std::string last;
  static uint64_t calls = 0;
  const char* e = std::getenv("PERM_FAULT");
  if (!e || !*e) return false;
  const std::string spec(e);
  const size_t colon = spec.find(':');
  const std::string name = spec.substr(0, colon);
  if (name != stage) return false;
  if (colon == std::string::npos) return true;
  const uint64_t k = std::strtoull(spec.c_str() + colon + 1, nullptr, 10);
  std::lock_guard<std::mutex> lk(mu);
  if (spec != last) {
    last = spec;
    calls = 0;
  }
  return ++calls == k;
}

void ensure_kernels_loaded() {
  static std::mutex mu;
  static std::atomic<bool> done[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  if (done[dev].load(std::memory_order_acquire)) return;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev].load(std::memory_order_relaxed)) return;
  for (int n = 1; n <= PERM_NMAX; ++n) {
    for (int c = 0; c < 2; ++c)
      for (int m = 0; m < 2; ++m)
        for (int r = 0; r < kRowModes; ++r)
          walk_resident_blocks(n, c != 0, m ? kProdF32 : kProdF64, (RowMode)r);  // loads the walk kernel
    if (n <= 32)
      mod_resident_lo(n);
    else if (n <= 48)
      mod_resident_mid(n);
    else
      mod_resident_hi(n);
  }
  batch_resident_blocks_rows(kRowsF64);
  batch_resident_blocks_rows(kRowsFixed);
  preload_abi_kernels();
  preload_batch_kernels();
  preload_mod_kernels();
  preload_peak_kernels();
  preload_ryser2_kernels();
  preload_sparse_kernels();
  preload_band_kernels();
  cudaGetLastError();
  done[dev].store(true, std::memory_order_release);
}

RowMode rows_from_env() {
  const char* e = std::getenv("PERM_ROWS");
  if (e && std::strcmp(e, "fp64") == 0) return kRowsF64;
  if (e && std::strcmp(e, "df") == 0) return kRowsDf;
  if (e && std::strcmp(e, "pair") == 0) return kRowsPair;
  if (e && std::strcmp(e, "fixed") == 0) return kRowsFixed;
  return kRowsPdf;  // FP64-product walks; the FP32-product ones take kRowsFixed
}

int pdf_tile_log() {
  const char* e = std::getenv("PERM_PDF_TILE_LOG");
  if (e && *e) {
    const int v = std::atoi(e);
    if (v >= 4 && v <= 16) return v;
  }
  return kPdfTileLog;
}

int walk_resident_blocks(int n, bool cplx, ProductMode mode, RowMode rows) {
  if (rows == kRowsDf && cplx && mode == kProdF64) return walk_blocks_df_c128(n);
  if (rows == kRowsPair && cplx && mode == kProdF64)
    return n <= 32 ? walk_blocks_xp_c128_lo(n) : walk_blocks_xp_c128_hi(n);
  if (rows == kRowsPdf && cplx && mode == kProdF64)
    return n <= 32 ? walk_blocks_pdf_c128_lo(n) : walk_blocks_pdf_c128_hi(n);
  if (rows == kRowsPdf && !cplx && mode == kProdF64)
    return n <= 32 ? walk_blocks_pdf_r64_lo(n) : walk_blocks_pdf_r64_hi(n);
  if (rows == kRowsDf || rows == kRowsPair || rows == kRowsPdf) rows = kRowsFixed;
  if (rows == kRowsFixed) {
    if (mode == kProdF64) {
      if (cplx) return n <= 32 ? walk_blocks_fx_c128_f64_lo(n) : walk_blocks_fx_c128_f64_hi(n);
      return walk_blocks_fx_r64_f64(n);
    }
    return cplx ? walk_blocks_fx_c128_f32(n) : walk_blocks_fx_r64_f32(n);
  }
  if (mode == kProdF64) {
    if (cplx) return n <= 32 ? walk_blocks_c128_f64_lo(n) : walk_blocks_c128_f64_hi(n);
    return walk_blocks_r64_f64(n);
  }
  return cplx ? walk_blocks_c128_f32(n) : walk_blocks_r64_f32(n);
}

cudaError_t walk_launch(bool cplx, ProductMode mode, const WalkArgs& a, RowMode rows) {
  if (rows == kRowsDf && cplx && mode == kProdF64) return walk_launch_df_c128(a);
  if (rows == kRowsPair && cplx && mode == kProdF64)
    return a.n <= 32 ? walk_launch_xp_c128_lo(a) : walk_launch_xp_c128_hi(a);
  if (rows == kRowsPdf && cplx && mode == kProdF64)
    return a.n <= 32 ? walk_launch_pdf_c128_lo(a) : walk_launch_pdf_c128_hi(a);
  if (rows == kRowsPdf && !cplx && mode == kProdF64)
    return a.n <= 32 ? walk_launch_pdf_r64_lo(a) : walk_launch_pdf_r64_hi(a);
  if (rows == kRowsDf || rows == kRowsPair || rows == kRowsPdf) rows = kRowsFixed;
  if (rows == kRowsFixed) {
    if (mode == kProdF64) {
      if (cplx) return a.n <= 32 ? walk_launch_fx_c128_f64_lo(a) : walk_launch_fx_c128_f64_hi(a);
      return walk_launch_fx_r64_f64(a);
    }
    return cplx ? walk_launch_fx_c128_f32(a) : walk_launch_fx_r64_f32(a);
  }
  if (mode == kProdF64) {
    if (cplx) return a.n <= 32 ? walk_launch_c128_f64_lo(a) : walk_launch_c128_f64_hi(a);
    return walk_launch_r64_f64(a);
  }
  return cplx ? walk_launch_c128_f32(a) : walk_launch_r64_f32(a);
}

}  // namespace perm

using namespace perm;

namespace {

constexpr int kMaxDevices = 64;

// Codes per launch: bounds each kernel to seconds at n ~ 40-48 on this part.
constexpr uint64_t kCodesPerLaunch = 1ull << 34;
// Minimum codes per thread before more threads are worth their seeding cost.
constexpr uint64_t kMinCodesPerThread = 16;

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return PERM_OK;
  if (e == cudaErrorMemoryAllocation) return PERM_ENOMEM;
  return PERM_ECUDA;
}

int current_device(int* dev) {
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= kMaxDevices) return PERM_ECUDA;
  return PERM_OK;
}

// True when p is memory the device can read directly (device or managed).
bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Scratch carved from one stream-ordered allocation.
struct Scratch {
  char* base = nullptr;
  cudaStream_t s = nullptr;
  ~Scratch() {
    if (base) cudaFreeAsync(base, s);
  }
  int alloc(size_t bytes, cudaStream_t stream) {
    s = stream;
    cudaError_t e = cudaMallocAsync((void**)&base, bytes ? bytes : 256, stream);
    if (e != cudaSuccess) {
      base = nullptr;
      cudaGetLastError();
      return status_of(e);
    }
    return PERM_OK;
  }
};

// Shared driver of every floating-point walk entry point.
//   final_mode 0: out = permanent (1 or 2 doubles); 1: out = dd partial.
int run_walk(bool cplx, ProductMode pm, const double* A, int n, uint64_t first, uint64_t count, int final_mode,
             double* out, void* stream_) {
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
  if (!A || !out) return PERM_ENULL;
  const uint64_t total = 1ull << (n - 1);
  if (first > total || count > total - first) return PERM_EINVAL;
  if (fault_injected("plan")) return PERM_ENOMEM;  // as if the scratch could not be had
  int dev = 0;
  int rc = current_device(&dev);
  if (rc) return rc;
  ensure_kernels_loaded();
  int* status = nullptr;
  rc = device_status_word(dev, &status);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream_;

  const int E = cplx ? 2 : 1;
  const size_t bytesA = (size_t)n * n * E * sizeof(double);
  const int out_doubles = final_mode == 0 ? E : 2 * E;
  const bool a_dev = is_device_ptr(A);
  const bool o_dev = is_device_ptr(out);

  const RowMode rows = rows_from_env();
  int resident = walk_resident_blocks(n, cplx, pm, rows);
  if (resident < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  uint64_t want = (count + kMinCodesPerThread * kWalkThreads - 1) / (kMinCodesPerThread * kWalkThreads);
  int blocks = (int)(want < 1 ? 1 : (want > (uint64_t)resident ? (uint64_t)resident : want));

  const size_t offA = 0, szA = a_dev ? 0 : align256(bytesA);
  const size_t offP = offA + szA, szP = align256((size_t)blocks * 2 * E * sizeof(double));
  const size_t offO = offP + szP, szO = o_dev ? 0 : align256(out_doubles * sizeof(double));
  Scratch scr;
  rc = scr.alloc(offO + szO, s);
  if (rc) return rc;
  const double* dA = A;
  if (!a_dev) {
    double* d = (double*)(scr.base + offA);
    cudaError_t e = cudaMemcpyAsync(d, A, bytesA, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return status_of(e);
    dA = d;
  }
  double* partials = (double*)(scr.base + offP);
  double* dOut = o_dev ? out : (double*)(scr.base + offO);

  if (fault_injected("launch")) return PERM_ECUDA;  // as if the walk's launch failed
  uint64_t done = 0;
  do {
    const uint64_t len = (count - done) < kCodesPerLaunch ? (count - done) : kCodesPerLaunch;
    WalkArgs a{dA, n, first + done, len, partials, blocks, done > 0 ? 1 : 0, status, s};
    cudaError_t e = walk_launch(cplx, pm, a, rows);
    if (e != cudaSuccess) return status_of(e);
    done += len;
  } while (done < count);

  if (fault_injected("finalize")) return PERM_ECUDA;  // the walk ran; its result is not delivered
  cudaError_t e = finalize_launch(partials, blocks, cplx, n, final_mode, dOut, s);
  if (e != cudaSuccess) return status_of(e);
  if (!o_dev) {
    e = cudaMemcpyAsync(out, dOut, out_doubles * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return status_of(e);
  }
  return PERM_OK;
}

}  // namespace

extern "C" {

int perm_c128(const double* A, int n, double* out, void* stream) {
  TraceRange trace("perm_c128");
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
  return run_walk(true, kProdF64, A, n, 0, 1ull << (n - 1), 0, out, stream);
}

int perm_f64(const double* A, int n, double* out, void* stream) {
  TraceRange trace("perm_f64");
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
  return run_walk(false, kProdF64, A, n, 0, 1ull << (n - 1), 0, out, stream);
}

int perm_c128_range(const double* A, int n, uint64_t first, uint64_t count, double* partial_dd, void* stream) {
  TraceRange trace("perm_c128_range");
  return run_walk(true, kProdF64, A, n, first, count, 1, partial_dd, stream);
}

int perm_f64_range(const double* A, int n, uint64_t first, uint64_t count, double* partial_dd, void* stream) {
  TraceRange trace("perm_f64_range");
  return run_walk(false, kProdF64, A, n, first, count, 1, partial_dd, stream);
}

int perm_c128_f32p(const double* A, int n, double* out, void* stream) {
  TraceRange trace("perm_c128_f32p");
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
  return run_walk(true, kProdF32, A, n, 0, 1ull << (n - 1), 0, out, stream);
}

int perm_f64_f32p(const double* A, int n, double* out, void* stream) {
  TraceRange trace("perm_f64_f32p");
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
  return run_walk(false, kProdF32, A, n, 0, 1ull << (n - 1), 0, out, stream);
}

int perm_last_status(void* stream) {
  int dev = 0;
  int rc = current_device(&dev);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  double limit = 86400.0;
  if (const char* env = std::getenv("PERM_TIMEOUT_S")) {
    double v = std::atof(env);
    if (v > 0) limit = v;
  }
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaStreamQuery(s);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return status_of(q);
    double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > limit) return PERM_ETIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  int* word = nullptr;
  rc = device_status_word(dev, &word);
  if (rc) return rc;
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, word, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return status_of(e);
  if (h) {
    e = cudaMemset(word, 0, sizeof(int));
    if (e != cudaSuccess) return status_of(e);
  }
  if (h & kStatusNonFinite) return PERM_ENONFINITE;
  return PERM_OK;
}

const char* perm_status_string(int st) {
  switch (st) {
    case PERM_OK: return "PERM_OK";
    case PERM_EINVAL: return "PERM_EINVAL: order or range out of bounds";
    case PERM_ENULL: return "PERM_ENULL: null pointer";
    case PERM_ECUDA: return "PERM_ECUDA: CUDA runtime error or no device";
    case PERM_ENONFINITE: return "PERM_ENONFINITE: non-finite input entry";
    case PERM_ETIMEOUT: return "PERM_ETIMEOUT: stream did not finish in time";
    case PERM_ENOMEM: return "PERM_ENOMEM: scratch allocation failed";
    case PERM_EPRIME: return "PERM_EPRIME: invalid modulus";
    default: return "unknown perm_status";
  }
}

void perm_shutdown(void) {
  batch_release_plans();
  int cur = -1, ndev = 0;
  cudaGetDevice(&cur);
  if (cudaGetDeviceCount(&ndev) == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_status_mu);
    for (int d = 0; d < ndev && d < kMaxDevices; ++d) {
      if (g_status_words[d] && cudaSetDevice(d) == cudaSuccess) {
        cudaFree(g_status_words[d]);
        g_status_words[d] = nullptr;
      }
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    }
  }
  if (cur >= 0) cudaSetDevice(cur);
  cudaGetLastError();
}

}  // extern "C"

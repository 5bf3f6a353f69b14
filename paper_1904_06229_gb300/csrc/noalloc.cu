// perm_c128_noalloc: the complex FP64 permanent for callers that must not
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaMallocAsync is not
// allowed or not wanted -- inside a host callback or a custom allocator's
// hook, under an application-wide memory budget that forbids allocations
// after start-up, or in a real-time loop that cannot afford the allocation's
// latency or possible synchronisation.  perm_c128 takes its per-block
// partial sums from a stream-ordered allocation on every call; this entry
// point takes them from one fixed array compiled into the library instead.
//
// The array is a file-scope static __device__ buffer of 2048 block slots
// (32 bytes each) plus 256 bytes for a status word: 65,792 bytes that every
// GPU which loads the library holds until the process exits.  A launch never
// uses more than 2048 blocks, so any order 1..PERM_NMAX fits; larger orders
// are rejected with PERM_EINVAL.  Host code cannot use the array's name as a
// device address, so the first call on each device (with that device
// current) looks the address up with cudaGetSymbolAddress and caches it; it
// also loads the library's kernels on that device.  That first call should
// therefore come before any stream capture or latency-critical use.
//
// Every call on a device shares the one array and leaves its contents behind:
// the status word is cleared by each call and the partial slots are
// overwritten before they are read.  Calls whose kernels overlap on the GPU
// (for example, on two streams at once) race on the array and give wrong
// results; serialise them.  A non-finite input entry makes the result NaN
// (perm_last_status does not see this entry point's status word).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "perm.h"
#include "perm_internal.h"

namespace {

constexpr int kNoAllocMaxBlocks = 2048;
constexpr int kNoAllocStatusDoubles = 32;  // 256 bytes; the status word lives at its start
constexpr size_t kNoAllocDoubles = (size_t)kNoAllocMaxBlocks * 4 + kNoAllocStatusDoubles;

static __device__ __align__(256) double g_perm_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDev = 64;
std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDev] = {nullptr};

constexpr uint64_t kNoAllocCodesPerLaunch = 1ull << 34;
constexpr uint64_t kNoAllocMinCodesPerThread = 16;

bool device_readable(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device address of the static array on the current device (looked up once).
int scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_perm_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return PERM_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return PERM_OK;
}

}  // namespace

extern "C" int perm_c128_noalloc(const double* A, int n, double* out, void* stream) {
  using namespace perm;
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
  if (!A || !out) return PERM_ENULL;
  int ndev = 0, dev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return PERM_ECUDA;
  // inputs and outputs must already be on the device: staging a host buffer
  // would need an allocation
  if (!device_readable(A) || !device_readable(out)) return PERM_EINVAL;
  // load every kernel of the library on this device first (once), so that no
  // launch below waits for a lazy module load behind running work
  ensure_kernels_loaded();
  double* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc) return rc;
  double* partials = scratch;
  int* status = reinterpret_cast<int*>(scratch + (size_t)kNoAllocMaxBlocks * 4);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  const RowMode rows = rows_from_env();  // the same kernel perm_c128 uses
  const int resident = walk_resident_blocks(n, true, kProdF64, rows);
  if (resident < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  const uint64_t count = 1ull << (n - 1);
  const uint64_t per_block = kNoAllocMinCodesPerThread * kWalkThreads;
  uint64_t want = (count + per_block - 1) / per_block;
  if (want < 1) want = 1;
  if (want > (uint64_t)resident) want = (uint64_t)resident;
  if (want > (uint64_t)kNoAllocMaxBlocks) want = kNoAllocMaxBlocks;
  const int blocks = (int)want;

  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e != cudaSuccess) return PERM_ECUDA;
  uint64_t done = 0;
  do {
    const uint64_t len = (count - done) < kNoAllocCodesPerLaunch ? (count - done) : kNoAllocCodesPerLaunch;
    WalkArgs a{A, n, done, len, partials, blocks, done > 0 ? 1 : 0, status, s};
    e = walk_launch(true, kProdF64, a, rows);
    if (e != cudaSuccess) return PERM_ECUDA;
    done += len;
  } while (done < count);
  e = finalize_launch(partials, blocks, true, n, 0, out, s);
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

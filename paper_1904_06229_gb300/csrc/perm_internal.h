// Internal host-side interfaces between the C ABI (perm_abi.cu) and the kernel
// translation units.  Not installed; the public surface is include/perm.h.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace perm {

// Device status bits (OR-ed into a per-device word by the kernels).
enum : int { kStatusNonFinite = 1 };

// Threads per block of the Gray-walk kernels.
constexpr int kWalkThreads = 128;

// Product arithmetic of a walk kernel.
enum ProductMode : int {
  kProdF64 = 0,  // FP64 products (Sec. 2.B "double")
  kProdF32 = 1,  // FP32 significands with integer exponents
};

// Row-sum arithmetic of a walk kernel.
enum RowMode : int {
  kRowsF64 = 0,    // FP64 row sums, DFMA updates, periodic re-seed (glynn_walk.cuh)
  kRowsFixed = 1,  // exact int64 fixed-point row sums, integer updates (glynn_walk_fx.cuh)
  kRowsDf = 2,     // double-float row sums and products on the FP32 pipe (glynn_walk_df.cuh);
                   // complex FP64-product walks only, the others use kRowsFixed
  kRowsPair = 3,   // exact float-pair row sums, packed double-float products (glynn_walk_xp.cuh);
                   // complex FP64-product walks only, the others use kRowsFixed
  kRowsPdf = 4,    // packed double-float row sums re-seeded from exact int64 and packed double-float
                   // products (glynn_walk_xp.cuh, glynn_walk_xr.cuh); FP64-product walks
};
constexpr int kRowModes = 5;

// Row arithmetic for the floating-point entry points: PERM_ROWS=fp64 selects
// kRowsF64, PERM_ROWS=df kRowsDf, PERM_ROWS=pair kRowsPair, PERM_ROWS=fixed
// kRowsFixed, anything else (default) kRowsPdf, which the walks without a
// packed variant (FP32-product, warp batch kernel) take as kRowsFixed.
RowMode rows_from_env();

// Re-seed period (log2 codes) of the packed double-float walk: PERM_PDF_TILE_LOG
// (4..16) or the default kPdfTileLog.
constexpr int kPdfTileLog = 10;
int pdf_tile_log();

struct WalkArgs {
  const double* A;     // device, row-major (interleaved re/im when complex)
  int n;               // order
  uint64_t first;      // first Gray code index of this launch
  uint64_t count;      // number of codes in this launch
  double* partials;    // blocks x (4 complex | 2 real) doubles: per-block dd sums
  int blocks;          // grid size (<= walk_resident_blocks)
  int accumulate;      // 1: add into partials, 0: overwrite
  int* status;         // device status word
  cudaStream_t stream;
};

// Largest useful grid for one walk launch (resident blocks on the device).
int walk_resident_blocks(int n, bool cplx, ProductMode mode, RowMode rows = kRowsF64);

// Launch the Gray-walk kernel for the given order / type / product / row mode.
cudaError_t walk_launch(bool cplx, ProductMode mode, const WalkArgs& a, RowMode rows = kRowsF64);

// Per-order dispatch inside each kernel translation unit.
cudaError_t walk_launch_c128_f64_lo(const WalkArgs& a);   // n in 1..32
cudaError_t walk_launch_c128_f64_hi(const WalkArgs& a);   // n in 33..64
cudaError_t walk_launch_r64_f64(const WalkArgs& a);       // n in 1..64
cudaError_t walk_launch_c128_f32(const WalkArgs& a);      // n in 1..64
cudaError_t walk_launch_r64_f32(const WalkArgs& a);       // n in 1..64
cudaError_t walk_launch_df_c128(const WalkArgs& a);  // double-float rows and products
int walk_blocks_df_c128(int n);
cudaError_t walk_launch_xp_c128_lo(const WalkArgs& a);  // exact float-pair rows, packed products, n in 1..32
cudaError_t walk_launch_xp_c128_hi(const WalkArgs& a);  // n in 33..64
int walk_blocks_xp_c128_lo(int n);
int walk_blocks_xp_c128_hi(int n);
cudaError_t walk_launch_pdf_r64_lo(const WalkArgs& a);   // the same for real matrices, n in 1..32
cudaError_t walk_launch_pdf_r64_hi(const WalkArgs& a);   // n in 33..64
int walk_blocks_pdf_r64_lo(int n);
int walk_blocks_pdf_r64_hi(int n);
cudaError_t walk_launch_pdf_c128_lo(const WalkArgs& a);  // packed double-float rows and products, n in 1..32
cudaError_t walk_launch_pdf_c128_hi(const WalkArgs& a);  // n in 33..64
int walk_blocks_pdf_c128_lo(int n);
int walk_blocks_pdf_c128_hi(int n);
cudaError_t walk_launch_fx_c128_f64_lo(const WalkArgs& a);  // fixed-point rows
cudaError_t walk_launch_fx_c128_f64_hi(const WalkArgs& a);
cudaError_t walk_launch_fx_r64_f64(const WalkArgs& a);
cudaError_t walk_launch_fx_c128_f32(const WalkArgs& a);
cudaError_t walk_launch_fx_r64_f32(const WalkArgs& a);
int walk_blocks_fx_c128_f64_lo(int n);
int walk_blocks_fx_c128_f64_hi(int n);
int walk_blocks_fx_r64_f64(int n);
int walk_blocks_fx_c128_f32(int n);
int walk_blocks_fx_r64_f32(int n);
int walk_blocks_c128_f64_lo(int n);
int walk_blocks_c128_f64_hi(int n);
int walk_blocks_r64_f64(int n);
int walk_blocks_c128_f32(int n);
int walk_blocks_r64_f32(int n);

// Fixed-order reduction of per-block dd partials.
//   mode 0: out = 2 (-1)^(n-1) * sum, rounded to double(s)  (1 or 2 doubles)
//   mode 1: out = sum as dd                                    (2 or 4 doubles)
//   mode 2: out = (-1)^n * sum, rounded to double(s)            (Ryser's un-halved form)
//   mode 3: out = 2^(1-n) * sum, rounded to double(s)           (Glynn's form with multiplicities)
cudaError_t finalize_launch(const double* partials, int nparts, bool cplx, int n, int mode, double* out,
                            cudaStream_t stream);

// ---- modular path ----
// Constants of the Montgomery walk (glynn_mod.cuh) for four odd moduli.
struct ModConsts {
  uint64_t p[4];
  uint64_t pinv[4];        // -p^-1 mod 2^64
  uint64_t r2[4];          // R^2 mod p, R = 2^64
  uint64_t fix[3][2][4];   // [G = 12, 8, 4][first group reduced through R^2, or not][q]: R^(groups - 1 + k) mod p
  uint64_t rpow[4][4];     // [w][q]: R^w mod p (w = 0..3), for reducing a 256-bit integer
  uint64_t pmin;           // smallest modulus
  int exact_ok;            // 0: always take the modular group walk (PERM_MOD_SUM=modular)
};
int mod_resident_lo(int n);   // n in 1..32
int mod_resident_mid(int n);  // n in 33..48
int mod_resident_hi(int n);   // n in 49..64
cudaError_t mod_launch_lo(int n, const int8_t* A, const ModConsts& c, uint64_t count, uint64_t* partials, int blocks,
                          cudaStream_t s);
cudaError_t mod_launch_mid(int n, const int8_t* A, const ModConsts& c, uint64_t count, uint64_t* partials, int blocks,
                           cudaStream_t s);
cudaError_t mod_launch_hi(int n, const int8_t* A, const ModConsts& c, uint64_t count, uint64_t* partials, int blocks,
                          cudaStream_t s);

// ---- batch path ----
constexpr int kBatchNMax = 32;  // largest order perm_batch accepts

// Kernel that walks the matrices of one order.
enum BatchKind : int {
  kBatchNone = 0,  // no matrices of this order
  kBatchWarp = 1,  // one warp per item, exact fixed-point rows (batch.cu: k_batch)
  kBatchCta = 2,   // one block of 128 threads per item, packed double-float walk, 255 registers (batch_cta.cu)
  kBatchCta3 = 3,  // the same with a 168-register cap (three blocks per SM)
  kBatchCta256 = 4,  // one block of 256 threads per item, one block per SM
};
constexpr int kBatchKinds = 5;
constexpr int kBatchCtaThreads = 128;  // threads of a block-per-item kernel

// Where the pointers of one call live: set by a one-thread kernel before each
// graph launch, so a cached plan serves any matrices and output of its shape.
struct BatchArgs {
  const double* const* ptrs;  // device array of `count` device matrix pointers
  double* out;                // 2 * count doubles
};

// Per-order layout of a batch (a kernel parameter).  Matrices are grouped by
// order, largest first (perm: positions -> matrix indices); the items of an
// order are (matrix slot, code chunk) pairs numbered slot-major.  Item
// partials are numbered by gbase; each kernel kind numbers its own items from
// 0 by kbase (its ticket space).
struct BatchTable {
  int kind[kBatchNMax + 1];
  int mstart[kBatchNMax + 1];  // first position of the order's matrices in perm
  int mcount[kBatchNMax + 1];  // matrices of the order
  uint64_t per_item[kBatchNMax + 1];          // codes per item
  uint64_t items_per_matrix[kBatchNMax + 1];  // ceil(2^(n-1) / per_item)
  uint64_t kbase[kBatchNMax + 1];             // first ticket of the order in its kernel
  uint64_t gbase[kBatchNMax + 1];             // first item partial of the order
  uint64_t kitems[kBatchKinds];               // tickets of each kernel kind
};

cudaError_t batch_launch_warp(const BatchArgs* ba, const int* perm, const BatchTable& tab, double* partials,
                              unsigned long long* ticket, int* status, RowMode rows, cudaStream_t s);
cudaError_t batch_launch_cta(int kind, const BatchArgs* ba, const int* perm, const BatchTable& tab, double* partials,
                             unsigned long long* ticket, int* status, cudaStream_t s);
int batch_resident_blocks_rows(RowMode rows);   // warp kernel
int batch_resident_blocks_cta(int kind);        // block-per-item kernels
// the two block-per-item variants (batch_cta2.cu, batch_cta3.cu)
cudaError_t batch_launch_cta_minb2(const BatchArgs* ba, const int* perm, const BatchTable& tab, int kind,
                                   double* partials, unsigned long long* ticket, int* status, cudaStream_t s);
cudaError_t batch_launch_cta_minb3(const BatchArgs* ba, const int* perm, const BatchTable& tab, int kind,
                                   double* partials, unsigned long long* ticket, int* status, cudaStream_t s);
int batch_resident_cta_minb2();
int batch_resident_cta_minb3();
cudaError_t batch_launch_cta256(const BatchArgs* ba, const int* perm, const BatchTable& tab, int kind,
                                double* partials, unsigned long long* ticket, int* status, cudaStream_t s);
int batch_resident_cta256();

// Per-device status word (device int, OR-ed by kernels; read and cleared by
// perm_last_status).  Allocated on first use.
int device_status_word(int dev, int** out);

// Drop the cached batch graphs and their buffers (perm_shutdown).
void batch_release_plans();

// ---- peak probe ----
cudaError_t pipe_probe_launch(int pipe, double* sink, int blocks, int iters, cudaStream_t stream);

// ---- tracing and host-side fault injection ----
// NVTX range named after a C ABI entry point, open for the duration of the
// host call (header-only NVTX: a no-op unless a profiler is attached).
class TraceRange {
 public:
  explicit TraceRange(const char* name);
  ~TraceRange();
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
// True when the environment variable PERM_FAULT names `stage` ("plan",
// "launch" or "finalize"): "stage" fails every call that reaches the step,
// "stage:k" only the k-th such call of the process (counted from the time
// the variable took its current value).  The caller then returns the error
// code the failing step would give, without touching the device.
bool fault_injected(const char* stage);

// ---- kernel loading ----
// CUDA loads kernels lazily by default, and loading a kernel waits until the
// device is idle: a kernel first launched behind running work would make that
// call block the host until the work is done.  Every entry point therefore
// loads all of the library's kernels on the current device once, before its
// first launch there (a few tens of milliseconds, once per device and process).
template <typename T>
inline void load_kernel(T* k) {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k);
}
void preload_abi_kernels();     // perm_abi.cu: the fixed-order finalize
void preload_batch_kernels();   // batch.cu: batch finalize and statistics
void preload_mod_kernels();     // glynn_mod.cu: modular finalize
void preload_peak_kernels();    // peak.cu: FP64 probe
void preload_ryser2_kernels();  // ryser2.cu
void preload_sparse_kernels();  // sparse.cu
void preload_band_kernels();    // band.cu
// Load every kernel on the current device (first call per device only; best
// effort: a kernel that fails to load here fails again at its launch, where
// the error is reported).
void ensure_kernels_loaded();

}  // namespace perm

/*
 * perm.h -- C ABI of the GB300 (sm_103a) permanent library `libperm.so`.
 *
 * The library computes matrix permanents (Eq. per of Lundow & Markstrom,
 * arXiv:1904.06229, Sec. 1) by the Gray-code ordered, halved inclusion-
 * exclusion sum of Sec. 2.A and Appendix A (Nijenhuis-Wilf / Glynn form of
 * Ryser's Eq. ryser):
 *
 *   per(A) = 2 (-1)^(n-1) sum_{r=0}^{2^(n-1)-1} (-1)^r prod_{i=1}^{n} w_i(x(r)),
 *   x(r)   = r xor (r >> 1)                   (Gray code of r, bit x_1 = LSB),
 *   w_i(x) = a_{i,n} - 1/2 sum_{j=1}^{n} a_{i,j} + sum_{j<n, x_j=1} a_{i,j}.
 *
 * Conventions shared by every entry point:
 *   - Matrices are n x n, row-major, densely packed.  Complex matrices are
 *     interleaved (re, im) doubles: 2*n*n doubles.
 *   - Unless stated otherwise a pointer may be device memory or host memory
 *     (pinned or pageable); host inputs are copied in and host outputs copied
 *     out on `stream`.  A host output is valid once `stream` has been
 *     synchronised.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Every compute call is asynchronous on `stream` and returns a
 *     perm_status at once: argument errors are reported before anything is
 *     launched; errors found on the device (non-finite input) are reported by
 *     perm_last_status().
 *   - The caller owns every buffer it passes.  The library allocates only
 *     per-call scratch (stream-ordered, released on `stream`) and one status
 *     word per device, released by perm_shutdown().
 *   - Results are deterministic for a given GPU model: partial sums are
 *     combined exactly (128-bit fixed-point integer sums of the per-thread
 *     double-doubles, independent of order) or in a fixed order, never with
 *     floating-point atomics.
 *   - The library never falls back to the CPU.  Without a CUDA device every
 *     compute call returns PERM_ECUDA.
 *   - Every compute call opens an NVTX range named after itself (visible in
 *     Nsight timelines; a no-op without a profiler).
 *   - For testing callers' error handling, the environment variable
 *     PERM_FAULT=plan|launch|finalize[:k] makes the walk entry points
 *     (perm_c128, perm_f64, their _range and _f32p forms) fail at that step
 *     -- plan: PERM_ENOMEM before any device work; launch: PERM_ECUDA before
 *     the walk is launched; finalize: PERM_ECUDA after the walk, with no
 *     result written -- on every call, or with ":k" only on the k-th call
 *     that reaches the step.  No device fault is involved.
 */
#ifndef PERM_H_
#define PERM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest supported order: the Gray index 0 <= r < 2^(n-1) is a uint64. */
#define PERM_NMAX 64

typedef enum {
  PERM_OK = 0,
  PERM_EINVAL = -1,     /* n < 1, n > PERM_NMAX, count < 0, range outside [0, 2^(n-1)) */
  PERM_ENULL = -2,      /* a required pointer is NULL */
  PERM_ECUDA = -3,      /* a CUDA runtime call failed (no device, launch failure, ...) */
  PERM_ENONFINITE = -4, /* an input entry was NaN or Inf (reported by perm_last_status) */
  PERM_ETIMEOUT = -5,   /* perm_last_status gave up waiting for the stream */
  PERM_ENOMEM = -6,     /* scratch allocation failed */
  PERM_EPRIME = -7      /* a modulus is even, < 3, >= 2^62, or repeated */
} perm_status;

/* ---- FP64 permanents (Sec. 2.A, App. A; precision scheme of Sec. 2.B) ----
 * Complex A (default row arithmetic): each row is scaled by a power of two
 * 2^G_i (max(sum_j |Re a_ij|, sum_j |Im a_ij|) 2^G_i < 1) and its row sum is
 * held as a double-float pair (two FP32 values, about 48 significant bits
 * relative to the sum itself), updated per Gray step by TwoSum/FastTwoSum on
 * the packed FP32 instructions of sm_100+ (two rows per instruction), and
 * re-seeded every 128 codes from its exact 64-bit integer value (entries
 * rounded once to 2^-61 of the row scale), so the step errors stay
 * independent.  The product of the n row sums is formed in double-float
 * (exact FP32 products by fused multiply-add, TwoSum sums) in four chains
 * renormalised by powers of two; each term is rebuilt as FP64.  Real A: the
 * same arithmetic with one component per row.  Each thread's terms are
 * summed in FP64 over runs of at most
 * 4096 codes and folded into a double-double accumulator; the per-thread
 * accumulators are added exactly as 128-bit fixed-point integers (per block,
 * then over the blocks) and converted once to double-double.  out: the
 * permanent, double-double rounded to double(s).
 * Observed error against the long-double oracle: about 1e-13 relative on
 * n = 40 and 48 Haar slices (within 1e-10 for every tested configuration);
 * the error grows with the sum's condition number sum|t| / |per|, which is
 * large for real Gaussian matrices (1e-10 from the exact walk at n = 36).
 * The environment variable PERM_ROWS selects another row arithmetic:
 * "fixed" (exact 64-bit fixed-point row sums; complex: about 0.85 n of the
 * factors multiplied in 64-bit integer block floating point, the rest in
 * FP64; real: FP64 products; about 1e-15 per term, 2.7x (complex) and 3.5x
 * (real) slower), "fp64" (FP64 row
 * sums restarted from their definition every 4096 codes), "df" (unpacked
 * double-float rows and products) or "pair" (exact float-pair row sums on a
 * 48-bit fixed grid: 1.4x faster than the default at n = 40, but the grid's
 * rounding of the entries is a fixed perturbation of the matrix, about 1e-11
 * relative at n = 40). */

/* Complex permanent. A: 2*n*n doubles (interleaved). out: 2 doubles (re, im). */
int perm_c128(const double* A, int n, double* out, void* stream);

/* Real permanent. A: n*n doubles. out: 1 double. */
int perm_f64(const double* A, int n, double* out, void* stream);

/* Partial Gray-code sum over the code range [first, first + count) of App. A
 * (the sum "subpermanent" computes for one part), without the final
 * 2 (-1)^(n-1) factor:
 *   partial = sum_{r=first}^{first+count-1} (-1)^r prod_i w_i(x(r)).
 * Requires first + count <= 2^(n-1).  count = 0 gives a zero partial.
 * partial_dd (complex): 4 doubles {re_hi, re_lo, im_hi, im_lo};
 * partial_dd (real):    2 doubles {hi, lo}.
 * Summing the partials of disjoint ranges that cover [0, 2^(n-1)) and
 * multiplying by 2 (-1)^(n-1) gives the permanent; this is how a long
 * computation is split across launches, streams, processes or GPUs, and how
 * it is checkpointed (state = next code index + partial). */
int perm_c128_range(const double* A, int n, uint64_t first, uint64_t count, double* partial_dd, void* stream);
int perm_f64_range(const double* A, int n, uint64_t first, uint64_t count, double* partial_dd, void* stream);

/* ---- Allocation-free variant of perm_c128 (the paper has no counterpart:
 * this exists for callers that cannot allocate device memory) ----
 * Same result as perm_c128 (same kernels, same summation order), for callers
 * that must not call cudaMalloc / cudaMallocAsync -- for example code running
 * in a host callback, inside an allocator hook, under a budget that forbids
 * allocation after start-up, or in a latency-bound loop.  The per-block
 * partial sums live in a fixed 65,792-byte static device array inside the
 * library (2048 block slots of 32 bytes plus a 256-byte status word), held by
 * every GPU that loads the library until the process exits; a launch never
 * uses more than 2048 blocks.  A and out must be DEVICE (or managed) memory:
 * host pointers are rejected with PERM_EINVAL, as are n < 1 and n > PERM_NMAX;
 * NULL gives PERM_ENULL.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) and must come before any stream
 * capture, and before any latency-critical use: it also loads the library's
 * kernels on that device (a few tens of milliseconds, once per device and
 * process).  All calls on a device share the array: calls whose kernels
 * overlap on the GPU (e.g. on two streams) race and must be serialised.  A
 * non-finite input gives a NaN result; perm_last_status does not report it
 * for this entry point.  The call itself allocates no memory. */
int perm_c128_noalloc(const double* A, int n, double* out, void* stream);

/* ---- FP32-product variant (precision schemes of Sec. 2.B: product precision
 * chosen apart from sum precision) ----
 * Row sums and the accumulation as in perm_c128 / perm_f64 (FP64, double-
 * double); each factor w_i is split into an integer power of two and an FP32
 * significand in [1, 2) (per term, by bit operations), the product of the n
 * significands is formed in FP32 and the exponents are added in integers; the
 * term is rebuilt as a double.  Relative error per term about n * 2^-24; the
 * result's error is reported against the FP64 oracle by the tests. */
int perm_c128_f32p(const double* A, int n, double* out, void* stream);
int perm_f64_f32p(const double* A, int n, double* out, void* stream);

/* ---- Repeated columns: the multiplicity classes of Eq.(ryser2), Sec. 2.A ----
 * For the n x n matrix A whose R distinct columns cbar_1..cbar_R appear m_k
 * times each (sum_k m_k = n; Boson-sampling outputs with several photons in
 * one mode give such matrices), the terms of the sum are grouped by
 * multiplicity as in Eq.(ryser2), but in Glynn's halved form (the form of
 * App. A), which is far better conditioned than the un-halved one:
 *   per(A) = 2^(1-n) sum_g (-1)^{sum g} C(m_1 - 1, g_1) prod_{k>1} C(m_k, g_k)
 *            prod_i sum_k (m_k - 2 g_k) cbar_k(i),
 * m_1 prod_{k>1} (m_k + 1) terms instead of 2^(n-1).
 * C: n x R complex matrix of the distinct columns, row-major interleaved
 *    (C[2*(i*R+k)] = Re cbar_k(i)); device or host memory.
 * mult: HOST array of R multiplicities >= 1 summing to n; 1 <= R <= n <= 64;
 *    at most 2^62 terms (PERM_EINVAL otherwise).
 * out: 2 doubles (re, im), device or host.  Row sums are exact int64 fixed
 * point, products as in perm_c128 (most factors in integer block floating
 * point, the rest in FP64), accumulation double-double; rows of A are not
 * merged (use the transpose for repeated rows: per(A) = per(A^T)). */
int perm_c128_repeated(const double* C, const int* mult, int R, int n, double* out, void* stream);

/* ---- Band matrices: the transfer-matrix recursion of App. C ("bandpermanent") ----
 * For A with a_ij = 0 whenever |i - j| > k: multiply the linear forms
 * C_i = sum_j a_ij x_j row by row with x_j^2 = 0, setting x_{i-k-1} = 1 once
 * no later row involves it, then all x = 1.  O(n 2^(2k+1) (2k+1)) work,
 * linear in n for fixed k; the kernel forms only the C(2k+1, k+1) window
 * subsets whose size a live monomial can have.
 * A: `count` complex n x n matrices, contiguous (count * 2*n*n doubles,
 *    row-major interleaved), device or host; only entries with |i - j| <= k
 *    are read (the others are taken as zero).
 * n: 1..65535; k: 0..5; 1 <= count <= 2^30, count * n * n <= 2^44
 * (PERM_EINVAL otherwise).  out: 2*count doubles (re, im), device
 * or host.  One CTA per matrix; the window polynomial (2^(2k+1) complex
 * coefficients) lives in shared memory; coefficients are formed in a fixed
 * order (deterministic). */
int perm_c128_band(const double* A, int n, int k, int count, double* out, void* stream);

/* ---- Sparse matrices: Ryser's sum restricted to dominating column sets
 * (Sec. 2.D, App. B "sparsepermanent" / "greedypartition") ----
 * A product prod_i sum_{j in J} a_ij is zero unless J meets the non-zero
 * columns of every row.  The greedy partition {S_1..S_d, T} of App. B (rows
 * of least out-degree first; best of 16 randomised tie-breaks by the number of
 * sets) restricts the sum to J = (non-empty subset of each S_l) u (any subset
 * of T): 2^|T| prod (2^|S_l| - 1) sets instead of 2^n.
 * A: complex n x n (interleaved, row-major), device or host; its non-zero
 * pattern is read on the host, so for a device A the call waits for `stream`
 * before returning (the walk itself is asynchronous).  n: 1..64.  out: 2
 * doubles.  PERM_EINVAL if the partition still has 2^63 sets or more. */
int perm_c128_sparse(const double* A, int n, double* out, void* stream);

/* The partition perm_c128_sparse uses, on the host (no GPU): block[j] = l for
 * column j in S_l, -1 for j in T; *count = number of sets (0 if >= 2^63). */
int perm_sparse_partition(const double* A_host, int n, int* block, uint64_t* count);

/* ---- Batch of independent complex permanents (the random-matrix studies of
 * Secs. 3-6 need 10^5..10^7 permanents of orders up to ~35) ----
 * ptrs: DEVICE array of `count` DEVICE pointers, each to a 2*n_k*n_k complex
 *       matrix; ns: HOST array of the `count` orders (1 <= n_k <= 32);
 * out:  DEVICE array of 2*count doubles (re, im per matrix).
 * The matrices are grouped by order, largest first, and each order's
 * (matrix, code chunk) work items go to one of three persistent kernels: one
 * warp per item with exact fixed-point rows, or one block of 128 threads per
 * item with the default packed double-float walk (128 threads allowing two
 * or three blocks per SM, or 256 threads); each kernel takes its items from
 * an atomic ticket,
 * and a last kernel adds each matrix's item partials in a fixed order.  The
 * kernel and the codes per thread of each order come from a per-GPU tuning
 * table (perm_batch_autotune, perm_batch_tuning); untuned orders take
 * built-in choices.  With PERM_ROWS=fixed or fp64 every order takes the
 * warp kernel with that row arithmetic.
 * The launches are captured in a CUDA graph (a plan) keyed by device,
 * stream, row arithmetic, the orders ns and the tuning; ptrs and out are
 * passed through a small device argument block set just before each graph
 * launch, so later calls with the same orders reuse the plan for any
 * matrices and output.  Building a plan allocates its buffers stream-ordered
 * on `stream` and uploads the order-sorted matrix positions through kernel
 * arguments: the call never waits for the device.  Up to 8 plans are kept;
 * dropping one (or perm_shutdown) frees its buffers with cudaFree, which
 * waits for launches still using them.  A plan holds at most 2^26 work items
 * (or one per matrix): larger batches get longer chunks for the orders with
 * the most items, so any batch size runs in one graph launch.  Results equal
 * perm_c128 on the same matrix with the same row arithmetic to within
 * rounding of the summation order. */
int perm_batch(const double* const* ptrs, const int* ns, int count, double* out, void* stream);

/* Number of batch plans built so far in this process (host only): a call
 * that reuses a cached plan leaves it unchanged. */
int perm_batch_plans(int* built);

/* ---- Batch with the random-matrix statistics of Secs. 3-6 ----
 * perm_batch, then, per order n = 0..32, statistics of X = |per(A)| / sqrt(n!)
 * over the batch's matrices of that order (the paper's normalisation, with
 * <X^2> = 1 for independent variance-1 entries):
 *   stats[n*PERM_STATS_STRIDE + 0]      number of matrices of order n
 *   stats[n*PERM_STATS_STRIDE + 1..4]   sum of X, X^2, X^3, X^4
 *   stats[n*PERM_STATS_STRIDE + 5 + b]  histogram, 16 bins per decade (Sec. 3):
 *       b = 0: X < 1e-4;  b = 1..96: 10^(-4+(b-1)/16) <= X < 10^(-4+b/16);
 *       b = 97: X >= 100.
 * stats: DEVICE array of 33 * PERM_STATS_STRIDE doubles (overwritten).
 * Chunks of 4096 results per block, then one block per order: the moment sums
 * are exact 128-bit fixed-point integer sums of per-thread FP64 sums (the same
 * value whatever the block order), counts are exact.  Per-call scratch of
 * about 450 bytes per chunk, stream-ordered.  10^7 results of one order take
 * about 1.5 ms on GB300. */
#define PERM_STATS_STRIDE 103
int perm_batch_stats(const double* const* ptrs, const int* ns, int count, double* out, double* stats, void* stream);

/* Fill the batch tuning table for orders n_lo..n_hi on the current device by
 * timing, per order, each kernel (warp per item; block of 128 threads per
 * item with up to 255 or 168 registers; block of 256 threads per item) at
 * each chunk length 16 .. 8192 codes per thread on
 * synthetic input (blocking, a few seconds).  Returns PERM_OK or an error. */
int perm_batch_autotune(int n_lo, int n_hi);

/* Batch kernel kinds of the tuning table. */
#define PERM_BATCH_WARP 1  /* one warp per item, exact fixed-point rows */
#define PERM_BATCH_CTA 2   /* one block of 128 threads per item, packed double-float walk, 2 blocks per SM */
#define PERM_BATCH_CTA3 3  /* the same with 3 blocks per SM (168 registers) */
#define PERM_BATCH_CTA256 4 /* one block of 256 threads per item, 1 block per SM */

/* Read (set = 0) or replace (set != 0) the batch tuning table of `device`
 * for the row arithmetic PERM_ROWS selects: L and kind are HOST arrays of 33
 * ints; for order n, kind[n] is the kernel (PERM_BATCH_*) and L[n] the codes
 * per thread (per lane for the warp kernel), both 0 when not tuned (index 0
 * unused).  On set every entry must be 0 in both arrays or a power of two in
 * 16 .. 2^24 with a kind 1..4 (PERM_EINVAL otherwise, nothing changed).
 * Host only: no CUDA call is made, so a table saved from one process can be
 * loaded into another before its first batch (the choices change only speed,
 * never results beyond rounding order). */
int perm_batch_tuning(int device, int* L, int* kind, int set);

/* ---- Exact permanents of small-integer matrices ----
 * Glynn's form (the App. A sum with v = 2w, an integer for integer A):
 *   2^(n-1) per(A) = (-1)^(n-1) sum_r (-1)^r prod_i v_i(x(r)),
 *   v_i(x) = 2 a_{i,n} - sum_j a_{i,j} + 2 sum_{j<n, x_j=1} a_{i,j},
 * evaluated modulo each of four odd primes below 2^62, then multiplied by
 * (-1)^(n-1) / 2^(n-1) mod p.  Row sums v_i are exact int32.  Where every
 * per-thread partial sum is provably below 2^255 (bound: codes per thread
 * times prod_i sum_j |a_ij|; 0-1 and +-1 matrices up to n of about 40), each
 * thread sums its terms exactly as a multi-limb integer and reduces that sum
 * modulo the primes once; otherwise exact products of row groups are combined
 * modulo each prime per term (64-bit Montgomery arithmetic).  The environment
 * variable PERM_MOD_SUM=modular forces the second form (same residues).  Any
 * odd moduli in [3, 2^62) give correct residues.
 * A: n*n int8 entries (any value, |a| <= 127).  primes: HOST array of 4
 * distinct odd moduli in [3, 2^62) (primality is the caller's promise; see
 * perm_default_primes).  residues: 4 uint64, per(A) mod primes[q] in [0, p).
 * Exact when |per(A)| < P/2, P = product of the moduli (about 2^247); the
 * sizes of 0-1 and +-1 matrices up to n = 64 satisfy this. */
int perm_mod01(const int8_t* A, int n, const uint64_t* primes, uint64_t* residues, void* stream);

/* Chinese remaindering on the host (no GPU): residues (k values, HOST) modulo
 * primes (k HOST values, pairwise coprime, product < 2^256) -> the unique x
 * with |x| <= P/2 congruent to them, as a 256-bit two's-complement integer in
 * out_limbs[4] (little-endian 64-bit limbs).  k in 1..4. */
int perm_crt(const uint64_t* residues, const uint64_t* primes, int k, uint64_t* out_limbs);

/* The four largest primes below 2^62 (deterministic Miller-Rabin search on
 * the host), in decreasing order. */
int perm_default_primes(uint64_t* out4);

/* ---- Status, measurement and teardown ---- */

/* Wait for `stream` (at most PERM_TIMEOUT_S seconds from the environment,
 * default 86400; PERM_ETIMEOUT if exceeded), then return and clear the first
 * error the device recorded since the last call (PERM_ENONFINITE), or
 * PERM_OK; PERM_ECUDA if the stream itself failed. */
int perm_last_status(void* stream);

/* Human-readable name of a perm_status value (static string). */
const char* perm_status_string(int status);

/* FP64 fused-multiply-add throughput of the current device, measured with
 * independent DFMA chains on every SM (blocking, about 0.1 s).  gops: lane
 * DFMA operations per second / 1e9 (one DFMA = 2 flops).  Same as
 * perm_pipe_peak(PERM_PIPE_DFMA, gops). */
int perm_fp64_peak(double* gops);

/* Instruction kinds of perm_pipe_peak. */
#define PERM_PIPE_DFMA 0  /* FP64 fused multiply-add, register operands */
#define PERM_PIPE_FFMA 1  /* FP32 fused multiply-add */
#define PERM_PIPE_FFMA2 2 /* packed FP32 fused multiply-add (two FMAs per lane instruction) */
#define PERM_PIPE_IMAD 3  /* 32-bit integer multiply-add */
#define PERM_PIPE_ALU 4   /* 32-bit three-input logic operation */
#define PERM_PIPE_ISSUE 5 /* packed FP32 FMAs and logic operations interleaved: the issue rate */

/* Throughput of one instruction kind on the current device: eight
 * independent chains per thread, 8 blocks of 256 threads per SM, best of five
 * timed launches (blocking, well under a second).  Not part of the method:
 * it measures the roofline denominators the walk kernels are compared with.
 * g_per_s: lane instructions per second / 1e9.  PERM_EINVAL for an unknown
 * kind, PERM_ENULL for a null pointer, PERM_ECUDA without a device,
 * PERM_ENOMEM if its 16 KB-per-SM sink cannot be allocated. */
int perm_pipe_peak(int pipe, double* g_per_s);

/* Free the library's per-device status words, cached graphs and the stream-
 * ordered memory pool's unused reserve.  Safe to call more than once; the
 * next compute call allocates afresh.  Call it with no work of the library in
 * flight, and launch no graph captured earlier from this library's calls
 * afterwards (such graphs hold the freed status word). */
void perm_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* PERM_H_ */

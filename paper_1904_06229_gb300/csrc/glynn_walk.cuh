// Gray-code walk kernel for the halved Ryser / Glynn sum (Sec. 2.A, App. A).
//
// One thread owns one contiguous range of Gray code indices (App. A
// "distribute" over all threads of the launch).  It seeds its row sums w_i
// directly from the code at the start of the range (App. A steps 2-8), then
// per code: forms p = prod_i w_i (step 10), adds (-1)^r p (steps 11-12), finds
// the flipped column j = ctz(r+1) and its direction (nextset, step 13) and
// updates every w_i by +-a_{i,j} (step 14).  The range is cut into runs that
// end at multiples of 2^12 codes; each run re-seeds w from its definition,
// which bounds the drift of the incremental updates, and its FP64 run sum is
// folded into a double-double accumulator (Sec. 2.B: compensated sum).
//
// Layout: A is staged once per block into shared memory column-major, so the
// column a step reads is contiguous and (when the lanes of a warp are at the
// same position inside their runs) a broadcast.  Row sums live in registers:
// the kernel is a template on the order N so every row index is a compile-
// time constant.
//
// GB300 note: FP64 FMA issues at about 2 lanes/clock/SM, 1/64 of FP32, so the
// kernel is bound by the FP64 pipe alone.  Every per-term operation that is
// not arithmetic on the row sums or products is kept off that pipe: the +-1
// factors are built from integer bits, row updates use one DFMA each (the
// DADD rate is lower than DFMA on this part), and the FP32-product mode
// rescales with integer bit operations instead of conversion instructions
// (which also run on the FP64 pipe).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include <cstdint>

#include "dd.cuh"
#include "perm_internal.h"

namespace perm {

constexpr int kRunLog = 12;
constexpr uint64_t kRun = 1ull << kRunLog;

template <int N, bool CPLX>
struct WalkShape {
  static constexpr int E = CPLX ? 2 : 1;  // doubles per entry
  static constexpr size_t smem_bytes = (size_t)(N * N + N) * E * sizeof(double) + 8 * sizeof(dd);
};

// 0.0 or 1.0 from a bit, integer operations only.
__device__ __forceinline__ double bit_to_double(uint32_t b) { return __hiloint2double((int)(b * 0x3FF00000u), 0); }

// ---- FP32 significand split (product mode kProdF32) ----
// Float with the bits of x scaled by 2^(1023 - e) (e = a biased FP64 exponent),
// mantissa rounded to 23 bits; 0 when x is zero, subnormal or scaled below
// the FP32 normal range.
__device__ __forceinline__ float scaled_f32(double x, int e) {
  uint32_t hi = (uint32_t)__double2hiint(x);
  uint32_t lo = (uint32_t)__double2loint(x);
  int ex = (int)((hi >> 20) & 0x7ff);
  int fexp = ex - e + 127;
  uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  uint32_t bits = (hi & 0x80000000u) | ((uint32_t)fexp << 23) | mant;
  bits += (lo >> 28) & 1u;  // round half up on the magnitude
  bool zero = (ex == 0) | (fexp <= 0);
  return __int_as_float(zero ? (int)(hi & 0x80000000u) : (int)bits);
}

// Double with value f * 2^E built from the bits of f (no conversion op).
__device__ __forceinline__ double f32_times_pow2(float f, int E) {
  uint32_t b = (uint32_t)__float_as_int(f);
  int fexp = (int)((b >> 23) & 0xff);
  int dexp = fexp - 127 + 1023 + E;
  uint32_t sign = b & 0x80000000u;
  uint32_t mant = b & 0x7FFFFFu;
  uint32_t hi = sign | ((uint32_t)dexp << 20) | (mant >> 3);
  uint32_t lo = mant << 29;
  if (fexp == 0 || dexp <= 0) hi = sign, lo = 0;
  if (dexp >= 2047) hi = sign | 0x7FF00000u, lo = 0;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ int dexp_of(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// ---- complex product of the row sums ----
// Four DFMAs with register operands only.  On GB300 a DFMA whose three
// operands are registers issues at 2 lanes/clk/SM, while DMUL, DADD and FMAs
// with a constant operand issue at 1.68; the two products are therefore
// written as FMAs onto `z`, a +-0.0 held in a register (the caller makes it
// from data, so it cannot be folded into a constant).
__device__ __forceinline__ void cmul(double& ar, double& ai, double br, double bi, double z) {
  double t = fma(ai, bi, z);
  double u = fma(ai, br, z);
  double nr = fma(ar, br, -t);
  double ni = fma(ar, bi, u);
  ar = nr;
  ai = ni;
}

__device__ __forceinline__ void cmulf(float& ar, float& ai, float br, float bi) {
  float t = ai * bi;
  float u = ai * br;
  float nr = fmaf(ar, br, -t);
  float ni = fmaf(ar, bi, u);
  ar = nr;
  ai = ni;
}

template <int N, bool CPLX, int MODE>
struct Product;

// FP64 products: two interleaved chains (even / odd rows) for ILP, N-1
// multiplies in all.
template <int N>
struct Product<N, true, kProdF64> {
  static __device__ __forceinline__ void eval(const double (&wr)[N], const double (&wi)[N], double& pr, double& pi,
                                              double z) {
    if constexpr (N == 1) {
      pr = wr[0];
      pi = wi[0];
    } else {
      double ar = wr[0], ai = wi[0], br = wr[1], bi = wi[1];
#pragma unroll
      for (int i = 2; i < N; i += 2) {
        cmul(ar, ai, wr[i], wi[i], z);
        if (i + 1 < N) cmul(br, bi, wr[i + 1], wi[i + 1], z);
      }
      cmul(ar, ai, br, bi, z);
      pr = ar;
      pi = ai;
    }
  }
};

template <int N>
struct Product<N, false, kProdF64> {
  static __device__ __forceinline__ void eval(const double (&w)[N], double& p, double z) {
    if constexpr (N == 1) {
      p = w[0];
    } else {
      double a = w[0], b = w[1];
#pragma unroll
      for (int i = 2; i < N; i += 2) {
        a = fma(a, w[i], z);
        if (i + 1 < N) b = fma(b, w[i + 1], z);
      }
      p = fma(a, b, z);
    }
  }
};

// FP32 significands: w_i = 2^(e_i - 1023) * (fr_i + i fi_i) with the larger
// component of each factor in [1, 2); |prod| lies in [1, 2^(1.5 N)) so the
// FP32 product never leaves the normal range.  Exponents add in integers.
template <int N>
struct Product<N, true, kProdF32> {
  static __device__ __forceinline__ void eval(const double (&wr)[N], const double (&wi)[N], double& pr, double& pi,
                                              double) {
    float ar = 1.f, ai = 0.f, br = 1.f, bi = 0.f;
    int E = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      int e = max(dexp_of(wr[i]), dexp_of(wi[i]));
      float fr = scaled_f32(wr[i], e);
      float fi = scaled_f32(wi[i], e);
      E += e - 1023;
      if (i == 0) {
        ar = fr, ai = fi;
      } else if (i == 1) {
        br = fr, bi = fi;
      } else if (i & 1) {
        cmulf(br, bi, fr, fi);
      } else {
        cmulf(ar, ai, fr, fi);
      }
    }
    if constexpr (N > 1) cmulf(ar, ai, br, bi);
    pr = f32_times_pow2(ar, E);
    pi = f32_times_pow2(ai, E);
  }
};

template <int N>
struct Product<N, false, kProdF32> {
  static __device__ __forceinline__ void eval(const double (&w)[N], double& p, double) {
    float a = 1.f, b = 1.f;
    int E = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      int e = dexp_of(w[i]);
      float f = scaled_f32(w[i], e);
      E += e - 1023;
      if (i & 1)
        b *= f;
      else
        a *= f;
    }
    p = f32_times_pow2(a * b, E);
  }
};

// Per-thread code range by the paper's "distribute" over all threads.
__device__ __forceinline__ void thread_range(uint64_t first, uint64_t count, uint64_t& r, uint64_t& end) {
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t q = count / T, rem = count % T;
  r = first + g * q + (g < rem ? g : rem);
  end = r + q + (g < rem ? 1 : 0);
}

// Flipped column and direction when moving from code r to r+1 (nextset):
// j = ctz(r+1); bit j of the new Gray code is 1 - bit (j+1) of r+1.
__device__ __forceinline__ void gray_step(uint64_t r, int& j, uint32_t& neg) {
  uint64_t r1 = r + 1;
  j = __ffsll((long long)r1) - 1;
  neg = (j < 63) ? (uint32_t)((r1 >> (j + 1)) & 1ull) : 0u;
}

// Stage A column-major into shared memory, compute w0_i = a_{i,N} - 1/2 sum_j a_ij
// (App. A step 5), report non-finite entries.
template <int N, bool CPLX>
__device__ __forceinline__ void stage(const double* __restrict__ A, double* sA, double* sW0, int* status) {
  constexpr int E = CPLX ? 2 : 1;
  int bad = 0;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
#pragma unroll
    for (int c = 0; c < E; ++c) {
      double v = A[(size_t)idx * E + c];
      bad |= not_finite(v) ? 1 : 0;
      sA[(j * N + i) * E + c] = v;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, (int)kStatusNonFinite);
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
#pragma unroll
    for (int c = 0; c < E; ++c) {
      double s = 0.0;
      for (int j = 0; j < N; ++j) s += sA[(j * N + i) * E + c];
      sW0[i * E + c] = fma(-0.5, s, sA[((N - 1) * N + i) * E + c]);
    }
  }
  __syncthreads();
}

// Block-level exact reduction of per-thread dd sums; thread 0 writes (or adds
// into) this block's slot of `partials`.
template <bool CPLX>
__device__ __forceinline__ void block_store_to(dd accr, dd acci, dd* sRed, double* o, int accumulate);

template <bool CPLX>
__device__ __forceinline__ void block_store(dd accr, dd acci, dd* sRed, double* partials, int accumulate) {
  block_store_to<CPLX>(accr, acci, sRed, partials + (size_t)blockIdx.x * (CPLX ? 4 : 2), accumulate);
}

// The same reduction, written to (or added into) the partial at o.  The
// threads' double-double sums are added exactly as 128-bit fixed-point
// integers (dd.cuh: fx128) on the integer pipes: the block's total does not
// depend on the order of the threads, and the FP64 pipe (1/64 of the FP32
// rate) converts only the one result.  A non-finite thread sum makes the
// partial NaN (the status word already records the non-finite input).
template <bool CPLX>
__device__ __forceinline__ void block_store_to(dd accr, dd acci, dd* sRed, double* o, int accumulate) {
  __shared__ int sEmax;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) sEmax = 1;
  __syncthreads();
  int e = max(dexp_field(accr.hi), dexp_field(accr.lo));
  if (CPLX) e = max(e, max(dexp_field(acci.hi), dexp_field(acci.lo)));
  e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
  if (lane == 0) atomicMax(&sEmax, e);
  __syncthreads();
  const int emax = sEmax;
  fx128* sF = reinterpret_cast<fx128*>(sRed);  // two fx128 per warp: the 32 bytes of two dd
  if (emax < 0x7FF) {
    const fx128 fr = fx128_warp_sum(fx128_add(fx128_of(accr.hi, emax), fx128_of(accr.lo, emax)));
    fx128 fi{0, 0};
    if (CPLX) fi = fx128_warp_sum(fx128_add(fx128_of(acci.hi, emax), fx128_of(acci.lo, emax)));
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
      const int nw = blockDim.x >> 5;
      for (int w = 1; w < nw; ++w) {
        fr = fx128_add(fr, sF[2 * w]);
        fi = fx128_add(fi, sF[2 * w + 1]);
      }
      tr = dd_of_fx128(fr, emax);
      ti = CPLX ? dd_of_fx128(fi, emax) : dd{0.0, 0.0};
    }
    if (accumulate) {
      tr = dd_add(tr, dd{o[0], o[1]});
      if (CPLX) ti = dd_add(ti, dd{o[2], o[3]});
    }
    o[0] = tr.hi;
    o[1] = tr.lo;
    if (CPLX) {
      o[2] = ti.hi;
      o[3] = ti.lo;
    }
  }
}

// Walk the codes [r, end) of one thread: seed, then per code product,
// signed accumulate, Gray step and row update (App. A steps 2-15).  The sum
// is added into the double-double accumulators.
template <int N, int MODE>
__device__ __forceinline__ void thread_walk_c128(const double2* __restrict__ sA2, const double2* __restrict__ sW02,
                                                 uint64_t r, const uint64_t end, dd& accr, dd& acci) {
  const double z = sA2[0].x * 0.0;  // a register zero (+-0.0) for the product FMAs
  double wr[N], wi[N];
  while (r < end) {
    const uint64_t run_end = min(end, (r | (kRun - 1)) + 1);
    // seed from the code of r (App. A steps 2, 5-8).  Rows are formed in a
    // rolled loop through a per-thread scratch array, so only one row sum
    // is live while it is being built.
    const uint64_t x = r ^ (r >> 1);
    {
      double2 seed[N];
#pragma unroll 1
      for (int i = 0; i < N; ++i) {
        double2 v = sW02[i];
#pragma unroll 1
        for (int j = 0; j < N - 1; ++j) {
          const double b = bit_to_double((uint32_t)(x >> j) & 1u);
          const double2 c = sA2[j * N + i];
          v.x = fma(b, c.x, v.x);
          v.y = fma(b, c.y, v.y);
        }
        seed[i] = v;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        wr[i] = seed[i].x;
        wi[i] = seed[i].y;
      }
    }
    double sr = 0.0, si = 0.0;
    uint32_t odd = (uint32_t)(r & 1ull);
    for (; r < run_end; ++r) {
      double pr, pi;
      Product<N, true, MODE>::eval(wr, wi, pr, pi, z);
      const double sg = pm_one(odd);
      odd ^= 1u;
      sr = fma(sg, pr, sr);
      si = fma(sg, pi, si);
      int j;
      uint32_t neg;
      gray_step(r, j, neg);
      const double dir = pm_one(neg);
      const double2* col = sA2 + j * N;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double2 c = col[i];
        wr[i] = fma(dir, c.x, wr[i]);
        wi[i] = fma(dir, c.y, wi[i]);
      }
    }
    accr = dd_add_d(accr, sr);
    acci = dd_add_d(acci, si);
  }
}

template <int N, int MODE>
__device__ __forceinline__ void thread_walk_r64(const double* __restrict__ sA, const double* __restrict__ sW0,
                                                uint64_t r, const uint64_t end, dd& accr) {
  const double z = sA[0] * 0.0;
  double w[N];
  while (r < end) {
    const uint64_t run_end = min(end, (r | (kRun - 1)) + 1);
    const uint64_t x = r ^ (r >> 1);
    {
      double seed[N];
#pragma unroll 1
      for (int i = 0; i < N; ++i) {
        double v = sW0[i];
#pragma unroll 1
        for (int j = 0; j < N - 1; ++j) v = fma(bit_to_double((uint32_t)(x >> j) & 1u), sA[j * N + i], v);
        seed[i] = v;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) w[i] = seed[i];
    }
    double s = 0.0;
    uint32_t odd = (uint32_t)(r & 1ull);
    for (; r < run_end; ++r) {
      double p;
      Product<N, false, MODE>::eval(w, p, z);
      s = fma(pm_one(odd), p, s);
      odd ^= 1u;
      int j;
      uint32_t neg;
      gray_step(r, j, neg);
      const double dir = pm_one(neg);
      const double* col = sA + j * N;
#pragma unroll
      for (int i = 0; i < N; ++i) w[i] = fma(dir, col[i], w[i]);
    }
    accr = dd_add_d(accr, s);
  }
}

template <int N, bool CPLX, int MODE>
__global__ void __launch_bounds__(kWalkThreads) k_walk(const double* __restrict__ A, uint64_t first, uint64_t count,
                                                       double* __restrict__ partials, int accumulate,
                                                       int* __restrict__ status) {
  constexpr int E = CPLX ? 2 : 1;
  extern __shared__ __align__(16) double smem[];
  double* sA = smem;
  double* sW0 = smem + N * N * E;
  dd* sRed = reinterpret_cast<dd*>(sW0 + N * E);

  stage<N, CPLX>(A, sA, sW0, status);

  uint64_t r, end;
  thread_range(first, count, r, end);

  dd accr{0.0, 0.0}, acci{0.0, 0.0};
  if constexpr (CPLX)
    thread_walk_c128<N, MODE>(reinterpret_cast<const double2*>(sA), reinterpret_cast<const double2*>(sW0), r, end,
                              accr, acci);
  else
    thread_walk_r64<N, MODE>(sA, sW0, r, end, accr);
  block_store<CPLX>(accr, acci, sRed, partials, accumulate);
}

// ---- host side: per-instantiation launch and occupancy ----
template <int N, bool CPLX, int MODE>
struct WalkKernel {
  static constexpr size_t smem = WalkShape<N, CPLX>::smem_bytes;

  static cudaError_t prepare(int& resident) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::atomic<int> cached[64];  // per device; filled once, read from any host thread
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (cached[dev] > 0) {
      resident = cached[dev];
      return cudaSuccess;
    }
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(k_walk<N, CPLX, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<N, CPLX, MODE>, kWalkThreads, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    cached[dev] = per_sm * sms;
    resident = cached[dev];
    return cudaSuccess;
  }

  static int resident_blocks() {
    int r = 0;
    return prepare(r) == cudaSuccess ? r : 0;
  }

  static cudaError_t launch(const WalkArgs& a) {
    int resident = 0;
    cudaError_t e = prepare(resident);
    if (e != cudaSuccess) return e;
    k_walk<N, CPLX, MODE><<<a.blocks, kWalkThreads, smem, a.stream>>>(a.A, a.first, a.count, a.partials,
                                                                      a.accumulate, a.status);
    return cudaGetLastError();
  }
};

template <bool CPLX, int MODE, int LO, int HI>
cudaError_t walk_dispatch(const WalkArgs& a) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    if (a.n == LO) return WalkKernel<LO, CPLX, MODE>::launch(a);
    return walk_dispatch<CPLX, MODE, LO + 1, HI>(a);
  }
}

template <bool CPLX, int MODE, int LO, int HI>
int walk_blocks_dispatch(int n) {
  if constexpr (LO > HI) {
    return 0;
  } else {
    if (n == LO) return WalkKernel<LO, CPLX, MODE>::resident_blocks();
    return walk_blocks_dispatch<CPLX, MODE, LO + 1, HI>(n);
  }
}

}  // namespace perm

// Double-double helpers (device), written from the published error-free
// transformations: Knuth's TwoSum and Dekker's FastTwoSum.  Only additions are
// used, so FMA contraction cannot alter them.  Used for the per-thread
// accumulator folds and the fixed-order reductions, never in the per-term path;
// block and grid totals are summed exactly as 128-bit fixed-point integers
// (fx128 below).
#pragma once

#include <cstdint>

namespace perm {

struct dd {
  double hi, lo;
};

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  e = __dsub_rn(b, __dsub_rn(s, a));
}

// dd + dd (the accurate variant: both halves through TwoSum).  Commutative
// bit-for-bit, so butterfly reductions give the same value on every lane.
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  double s1, s2, t1, t2;
  two_sum(a.hi, b.hi, s1, s2);
  two_sum(a.lo, b.lo, t1, t2);
  s2 = __dadd_rn(s2, t1);
  fast_two_sum(s1, s2, s1, s2);
  s2 = __dadd_rn(s2, t2);
  fast_two_sum(s1, s2, s1, s2);
  return dd{s1, s2};
}

// dd + double
__device__ __forceinline__ dd dd_add_d(dd a, double b) {
  double s, e;
  two_sum(a.hi, b, s, e);
  e = __dadd_rn(e, a.lo);
  fast_two_sum(s, e, s, e);
  return dd{s, e};
}

// ---- Exact sums of double-double values on the integer pipes ----
// A set of doubles is summed as signed 128-bit fixed-point integers in units
// of 2^(emax - 1075 - kFxFrac), emax the largest biased exponent in the set
// (at least 1).  Each double converts exactly apart from its bits below that
// unit (below 2^-108 of the largest value); integer addition is exact and
// associative, so the sum is the same for every order and tree, and no FP64
// instruction runs until the one conversion back (a double-double tree would
// issue 20 FP64 instructions per addition, on a pipe with 1/64 of the FP32
// rate here).  Headroom: each value is below 2^(53 + kFxFrac) units and at
// most 2^13 values are summed, so every partial sum stays below 2^122.
constexpr int kFxFrac = 56;

struct fx128 {
  long long h;          // high 64 bits (signed)
  unsigned long long l;  // low 64 bits
};

// Biased exponent field of a double (0 for zero and subnormals, 0x7FF for
// infinities and NaN).
__device__ __forceinline__ int dexp_field(double d) {
  return (int)(((unsigned long long)__double_as_longlong(d) >> 52) & 0x7FFull);
}

// d in units of 2^(emax - 1075 - kFxFrac), magnitude truncated; requires
// dexp_field(d) <= emax, 1 <= emax < 0x7FF.
__device__ __forceinline__ fx128 fx128_of(double d, int emax) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
  const int E = (int)((bits >> 52) & 0x7FFull);
  unsigned long long M = bits & 0xFFFFFFFFFFFFFull;
  int e = 1;  // subnormals: no implicit bit, the exponent of the smallest normal
  if (E != 0) {
    M |= 1ull << 52;
    e = E;
  }
  const int sh = e - emax + kFxFrac;  // <= kFxFrac < 64
  unsigned long long hi = 0, lo = 0;
  if (sh > 0) {
    lo = M << sh;
    hi = M >> (64 - sh);
  } else if (sh > -64) {
    lo = M >> (-sh);
  }
  if (bits >> 63) {  // two's complement negation of (hi, lo)
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  return fx128{(long long)hi, lo};
}

__device__ __forceinline__ fx128 fx128_add(fx128 a, fx128 b) {
  const unsigned long long l = a.l + b.l;
  return fx128{a.h + b.h + (l < a.l ? 1ll : 0ll), l};
}

__device__ __forceinline__ fx128 fx128_warp_sum(fx128 a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    const fx128 b{__shfl_xor_sync(0xffffffffu, a.h, m), __shfl_xor_sync(0xffffffffu, a.l, m)};
    a = fx128_add(a, b);
  }
  return a;
}

// Round to nearest (ties to even) of the unsigned 128-bit integer (mh, ml)
// times 2^ex, with integer instructions only: the double's magnitude bits, and
// the remainder m - RN(m) in units of 2^ex as a sign and a 128-bit magnitude.
// False when the double would not be normal.
__device__ __forceinline__ bool u128_rn(unsigned long long mh, unsigned long long ml, int ex,
                                        unsigned long long& bits, unsigned& rneg, unsigned long long& rh,
                                        unsigned long long& rl) {
  rneg = 0;
  rh = rl = 0;
  if ((mh | ml) == 0) {
    bits = 0;
    return true;
  }
  const int L = mh ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);  // bit length
  unsigned long long mant;
  int s = L - 53;  // the 53-bit significand is m 2^-s
  if (s <= 0) {
    mant = ml << (-s);  // exact
  } else {
    unsigned long long remh, reml, hh, hl, th, tl;
    if (s >= 64) {
      mant = mh >> (s - 64);
      remh = s > 64 ? mh & ((1ull << (s - 64)) - 1) : 0;
      reml = ml;
      th = 1ull << (s - 64);
      tl = 0;
    } else {
      mant = (mh << (64 - s)) | (ml >> s);
      remh = 0;
      reml = ml & ((1ull << s) - 1);
      th = 0;
      tl = 1ull << s;
    }
    if (s - 1 >= 64) {
      hh = 1ull << (s - 65);
      hl = 0;
    } else {
      hh = 0;
      hl = 1ull << (s - 1);
    }
    const bool gt = remh > hh || (remh == hh && reml > hl);
    const bool eq = remh == hh && reml == hl;
    if (gt || (eq && (mant & 1ull))) {  // round up: the remainder is rem - 2^s
      ++mant;
      rneg = 1;
      rl = tl - reml;
      rh = th - remh - (tl < reml ? 1ull : 0ull);
    } else {
      rh = remh;
      rl = reml;
    }
    if (mant == (1ull << 53)) {
      mant >>= 1;
      ++s;
    }
  }
  const int biased = 1075 + s + ex;
  if (biased < 1 || biased > 2046) return false;
  bits = ((unsigned long long)biased << 52) | (mant & ((1ull << 52) - 1));
  return true;
}

// The fixed-point value v (units 2^(emax - 1075 - kFxFrac + extra)) as the
// double-double (RN(v), RN(v - RN(v))), with integer instructions; values
// outside the normal double range take an FP64 route instead (v = h 2^64 + l
// split into four exact doubles, summed in order, scaled by scalbn).
__device__ __forceinline__ dd dd_of_fx128(fx128 v, int emax, int extra = 0) {
  const int ex = emax - 1075 - kFxFrac + extra;
  unsigned long long h = (unsigned long long)v.h, l = v.l;
  const unsigned neg = (unsigned)(h >> 63);
  if (neg) {
    l = ~l + 1ull;
    h = ~h + (l == 0ull ? 1ull : 0ull);
  }
  unsigned long long hb, lb, rh, rl, t1, t2;
  unsigned rneg, t0;
  if (u128_rn(h, l, ex, hb, rneg, rh, rl) && u128_rn(rh, rl, ex, lb, t0, t1, t2)) {
    const double hi = __longlong_as_double((long long)(hb | ((unsigned long long)neg << 63)));
    const double lo = lb ? __longlong_as_double((long long)(lb | ((unsigned long long)(neg ^ rneg) << 63))) : 0.0;
    return dd{hi, lo};
  }
  const double ph = __ll2double_rn(v.h);  // |v.h| < 2^58: the conversion back is exact
  const long long rh2 = v.h - __double2ll_rn(ph);
  dd r{ph * 0x1p64, 0.0};
  r = dd_add_d(r, (double)rh2 * 0x1p64);
  r = dd_add_d(r, __ull2double_rn(v.l & ~0x7FFull));
  r = dd_add_d(r, __ull2double_rn(v.l & 0x7FFull));
  return dd{scalbn(r.hi, ex), scalbn(r.lo, ex)};
}

// Exact sum over the 32 lanes of a warp of each lane's double-double: fx128
// in units of the warp's largest exponent, converted back once (times
// 2^extra); every lane returns the same total (NaN if any lane holds a
// non-finite value).
__device__ __forceinline__ dd dd_warp_sum_exact(dd a, int extra = 0) {
  int e = max(dexp_field(a.hi), dexp_field(a.lo));
  e = max(1, (int)__reduce_max_sync(0xffffffffu, (unsigned)e));
  if (e >= 0x7FF) return dd{__longlong_as_double(0x7ff8000000000000ll), 0.0};
  const fx128 f = fx128_warp_sum(fx128_add(fx128_of(a.hi, e), fx128_of(a.lo, e)));
  return dd_of_fx128(f, e, extra);
}

// +-1.0 from a bit, built with integer operations only (no FP64 instruction).
__device__ __forceinline__ double pm_one(uint32_t negative) {
  return __hiloint2double((int)(0x3FF00000u | (negative << 31)), 0);
}

// Flip the sign of a double with an integer XOR on its high word.
__device__ __forceinline__ double flip_sign(double x, uint32_t negative) {
  int hi = __double2hiint(x) ^ (int)(negative << 31);
  return __hiloint2double(hi, __double2loint(x));
}

// Non-finite test on the bit pattern (exponent field all ones).
__device__ __forceinline__ bool not_finite(double x) {
  return ((__double2hiint(x) >> 20) & 0x7ff) == 0x7ff;
}

}  // namespace perm

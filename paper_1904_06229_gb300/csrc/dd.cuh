// Double-double helpers (device), written from the published error-free
// transformations: Knuth's TwoSum and Dekker's FastTwoSum.  Only additions are
// used, so FMA contraction cannot alter them.  Used for the per-thread
// accumulator folds and the fixed-order reductions, never in the per-term path.
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

__device__ __forceinline__ dd dd_shfl_xor(dd a, int mask) {
  return dd{__shfl_xor_sync(0xffffffffu, a.hi, mask), __shfl_xor_sync(0xffffffffu, a.lo, mask)};
}

// Butterfly reduction of a dd over the 32 lanes of a warp (fixed tree).
__device__ __forceinline__ dd dd_warp_sum(dd a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) a = dd_add(a, dd_shfl_xor(a, m));
  return a;
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

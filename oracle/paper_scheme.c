/*
 * ORACLE DIRECTORY -- test and benchmark infrastructure only.
 *
 * The paper's own CPU scheme for the Gray-code permanent, as a second CPU
 * baseline for the benchmark (not a reference for parity: the long-double
 * oracle in perm_oracle.c is that).  Sec. 2.B evaluates the sum in plain
 * double precision with Kahan summation of the terms, the work split into
 * consecutive parts by App. A "distribute" and run in parallel, the partial
 * sums kept in an array and added in a fixed order.  This file follows that
 * description: double row sums w_i updated once per Gray step (App. A steps
 * 13-14), the product of the w_i in double (step 10), the signed term added
 * with Kahan's compensated summation (step 12 and the Kahan listing of
 * Sec. 2.B), OpenMP over the parts.  Only the benchmark's CPU-baseline leg
 * loads it; it shares nothing with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PS_NMAX 64

/* Kahan's summation: s accumulates, c carries the lost low part. */
typedef struct {
  double s, c;
} kahan;

static void kahan_add(kahan* k, double x) {
  double y = x - k->c;
  double t = k->s + y;
  k->c = (t - k->s) - y;
  k->s = t;
}

/* sum over r in [first, first + count) of (-1)^r prod_i w_i(gray(r)), with
 * w_i = a_{i,n} - 1/2 sum_j a_ij + sum_{j<n, x_j = 1} a_ij, in double. */
static void ps_range(const double* A, int n, uint64_t first, uint64_t count, double* re, double* im) {
  double wr[PS_NMAX], wi[PS_NMAX];
  const uint64_t x0 = first ^ (first >> 1);
  for (int i = 0; i < n; ++i) {
    double sr = 0, si = 0;
    for (int j = 0; j < n; ++j) sr += A[2 * (i * n + j)], si += A[2 * (i * n + j) + 1];
    wr[i] = A[2 * (i * n + n - 1)] - 0.5 * sr;
    wi[i] = A[2 * (i * n + n - 1) + 1] - 0.5 * si;
    for (int j = 0; j < n - 1; ++j)
      if ((x0 >> j) & 1) wr[i] += A[2 * (i * n + j)], wi[i] += A[2 * (i * n + j) + 1];
  }
  kahan kr = {0, 0}, ki = {0, 0};
  for (uint64_t k = 0; k < count; ++k) {
    const uint64_t r = first + k;
    double pr = wr[0], pi = wi[0];
    for (int i = 1; i < n; ++i) {
      const double nr = pr * wr[i] - pi * wi[i];
      const double ni = pr * wi[i] + pi * wr[i];
      pr = nr, pi = ni;
    }
    if (r & 1) pr = -pr, pi = -pi;
    kahan_add(&kr, pr);
    kahan_add(&ki, pi);
    /* Gray step r -> r + 1: column j = ctz(r + 1) flips; it becomes set
     * (+a) when bit j + 1 of r + 1 is 0, cleared (-a) otherwise. */
    const uint64_t r1 = r + 1;
    const int j = __builtin_ctzll(r1);
    if (j >= n - 1) continue; /* past the last code of the whole walk */
    const double z = ((r1 >> (j + 1)) & 1) ? -1.0 : 1.0;
    for (int i = 0; i < n; ++i) wr[i] += z * A[2 * (i * n + j)], wi[i] += z * A[2 * (i * n + j) + 1];
  }
  *re = kr.s;
  *im = ki.s;
}

/* The same sum over [first, first + count), split into `parts` consecutive
 * pieces (App. A distribute) evaluated in parallel on `threads` threads (0:
 * the OpenMP default); the partials are added in piece order with Kahan's
 * summation.  out: {re, im}.  Returns 0, or -1 for bad arguments. */
int paper_scheme_range(const double* A, int n, uint64_t first, uint64_t count, int parts, int threads,
                       double* out) {
  if (n < 1 || n > PS_NMAX || !A || !out || parts < 1) return -1;
  const uint64_t total = 1ull << (n - 1);
  if (first > total || count > total - first) return -1;
  if ((uint64_t)parts > count && count > 0) parts = (int)count;
  double* part = (double*)calloc((size_t)parts * 2, sizeof(double));
  if (!part) return -1;
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(static, 1) num_threads(threads)
#endif
  for (int k = 0; k < parts; ++k) {
    const uint64_t q = count / (uint64_t)parts, rem = count % (uint64_t)parts;
    const uint64_t s = first + (uint64_t)k * q + ((uint64_t)k < rem ? (uint64_t)k : rem);
    const uint64_t l = q + ((uint64_t)k < rem ? 1 : 0);
    ps_range(A, n, s, l, &part[2 * k], &part[2 * k + 1]);
  }
  kahan kr = {0, 0}, ki = {0, 0};
  for (int k = 0; k < parts; ++k) kahan_add(&kr, part[2 * k]), kahan_add(&ki, part[2 * k + 1]);
  free(part);
  out[0] = kr.s;
  out[1] = ki.s;
  return 0;
}

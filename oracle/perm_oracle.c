/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously-correct CPU reference for the matrix permanent of
 * Lundow & Markstrom, "Efficient computation of permanents, with applications
 * to Boson sampling and random matrices" (arXiv:1904.06229).  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load this
 * library.  It shares no code, header, table or constant with the CUDA library
 * in the package; the two are checked against each other, never against
 * themselves.
 *
 * Contents (each function cites the passage it follows):
 *   oracle_per_brute_c   Eq.(per): sum over all n! permutations (n <= 10).
 *   oracle_per_ryser_c   Eq.(ryser): Ryser's inclusion-exclusion over all 2^n
 *                        subsets J, row sums recomputed from scratch (n <= 24).
 *   oracle_glynn_part_c  App. A "subpermanent": Gray-code walk over a range of
 *                        code indices, steps in the paper's order (distribute,
 *                        unrank, nextset, the w update), long double arithmetic
 *                        with Neumaier-compensated accumulation.
 *   oracle_per_glynn_c   App. A "permanent": m parts (OpenMP over parts),
 *                        partials kept in an array and summed in fixed order
 *                        with compensation (Sec. 2.B), scaled by 2(-1)^n.
 *   oracle_glynn_exact_i8  exact integer form of the same sum (512-bit signed
 *                        integers), for integer matrices.
 *   oracle_glynn_mod_i8  the same sum modulo 64-bit primes, products reduced
 *                        with unsigned __int128 division.
 *   oracle_ryser2_c      Eq.(ryser2): the weighted Ryser sum for a matrix with
 *                        repeated columns, over all multiplicity vectors f,
 *                        row sums formed from scratch for every f.
 *   oracle_sparse_c      App. B "sparsepermanent": Ryser's sum restricted to
 *                        the sets J that meet every block S_l of a partition
 *                        {S_1..S_d, T} (non-empty subset of each S_l, any
 *                        subset of T), row sums formed from scratch.
 *
 * Real matrices are complex matrices with zero imaginary part; every function
 * takes an interleaved (re, im) row-major n x n array of doubles.
 *
 * Conventions (App. A): columns and Gray bits are 1-based in the comments and
 * 0-based in code; bit x_1 is the least significant bit of the unranked code
 * (nextset starts its scan at the first position).  Code index r carries the
 * sign t = (-1)^(r+1) because nextset flips t before the term is added.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double ld;

#define ORACLE_NMAX 64

/* Planted mistakes for the mutation test of the pins (tests/test_oracle_mutants.py
 * compiles this file with -DORACLE_MUTANT=k, k = 1..6; the normal build has 0):
 * 1 drops the last row from each product, 2 never flips the sign t, 3 seeds w
 * with the first column instead of the last, 4 reads the updated column
 * transposed, 5 forgets the halving in step 5, 6 uses the wrong final sign. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUT(k) (ORACLE_MUTANT == (k))

/* ---- Neumaier's variant of Kahan summation (Sec. 2.B recommends Kahan; the
 * Neumaier form also handles terms larger than the running sum). ---------- */
typedef struct {
  ld s, c;
} csum;

static void csum_add(csum* a, ld x) {
  ld t = a->s + x;
  if (fabsl(a->s) >= fabsl(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

static ld csum_value(const csum* a) { return a->s + a->c; }

#define RE(A, n, i, j) ((ld)(A)[2 * ((size_t)(i) * (n) + (j))])
#define IM(A, n, i, j) ((ld)(A)[2 * ((size_t)(i) * (n) + (j)) + 1])

/* ---- Eq.(per): brute force over permutations (Heap's algorithm) -------- */
int oracle_per_brute_c(const double* A, int n, ld* out /* re, im */) {
  if (n < 1 || n > 10 || !A || !out) return -1;
  int perm[10], c[10];
  for (int i = 0; i < n; ++i) perm[i] = i, c[i] = 0;
  csum sr = {0, 0}, si = {0, 0};
  for (;;) {
    /* product over rows i of a_{i, pi(i)} */
    ld pr = 1, pi = 0;
    for (int i = 0; i < n; ++i) {
      ld ar = RE(A, n, i, perm[i]), ai = IM(A, n, i, perm[i]);
      ld nr = pr * ar - pi * ai, ni = pr * ai + pi * ar;
      pr = nr, pi = ni;
    }
    csum_add(&sr, pr);
    csum_add(&si, pi);
    /* next permutation (Heap, iterative) */
    int i = 1;
    while (i < n && c[i] >= i) c[i] = 0, ++i;
    if (i >= n) break;
    int k = (i % 2 == 0) ? 0 : c[i];
    int t = perm[k];
    perm[k] = perm[i];
    perm[i] = t;
    ++c[i];
  }
  out[0] = csum_value(&sr);
  out[1] = csum_value(&si);
  return 0;
}

/* ---- Eq.(ryser): per(A) = (-1)^n sum_{J subset N} (-1)^{|J|} prod_i sum_{j in J} a_ij.
 * Every subset is visited in plain binary order and its row sums are formed
 * from scratch: no Gray code, no halving. ------------------------------- */
int oracle_per_ryser_c(const double* A, int n, ld* out) {
  if (n < 1 || n > 24 || !A || !out) return -1;
  csum sr = {0, 0}, si = {0, 0};
  uint64_t nsub = 1ull << n;
  for (uint64_t J = 0; J < nsub; ++J) {
    ld pr = 1, pi = 0;
    for (int i = 0; i < n; ++i) {
      ld rr = 0, ri = 0;
      for (int j = 0; j < n; ++j)
        if (J >> j & 1) rr += RE(A, n, i, j), ri += IM(A, n, i, j);
      ld nr = pr * rr - pi * ri, ni = pr * ri + pi * rr;
      pr = nr, pi = ni;
    }
    int sign = (__builtin_popcountll(J) & 1) ? -1 : 1;
    csum_add(&sr, sign * pr);
    csum_add(&si, sign * pi);
  }
  ld s = (n & 1) ? -1 : 1;
  out[0] = s * csum_value(&sr);
  out[1] = s * csum_value(&si);
  return 0;
}

/* ---- App. A "distribute(n, m, i, k, l)": split a sequence of length total
 * into m nearly equal consecutive pieces; piece i starts at k, has length l. */
static void distribute(uint64_t total, uint64_t m, uint64_t i, uint64_t* k, uint64_t* l) {
  uint64_t q = total / m;
  uint64_t r = total % m;
  *k = i * q + (i < r ? i : r);
  *l = q + (i < r ? 1 : 0);
}

/* ---- App. A unrank: the k-th Gray code is xor(k, rshift(k)); x[1] is its
 * least significant bit.  x has room for positions 1..n. --------------- */
static void unrank(uint64_t k, int n, int* x) {
  uint64_t g = k ^ (k >> 1);
  for (int j = 1; j <= n; ++j) x[j] = (j <= 64) ? (int)((g >> (j - 1)) & 1) : 0;
}

/* ---- App. A "nextset(t, j, x)": flip t; if t is now +1, scan from the first
 * position to the first set bit of x and move one past it; else take the
 * first position.  Then toggle x_j.  Returns j (1-based). --------------- */
static int nextset(int* t, int* x, int n) {
  int j = 1;
  if (!MUT(2)) *t = -*t;
  if (*t == 1) {
    while (j <= n && x[j] == 0) ++j;
    j = j + 1;
  }
  /* the final code of the whole sequence moves to position n, one past the
   * n-1 Gray positions; x has room for it and the update it drives is never
   * used (the walk ends). */
  if (j > n) j = n;
  x[j] = 1 - x[j];
  return j;
}

/* ---- App. A "subpermanent" generalised to an explicit range of code indices
 * [first, first + count): S = sum over the range of t * prod_i w_i with the
 * paper's sign t.  Also returns sum |t * prod w| (for a condition number). */
int oracle_glynn_range_c(const double* A, int n, uint64_t first, uint64_t count, ld* out /* re, im */,
                         ld* abs_sum) {
  if (n < 1 || n > ORACLE_NMAX || !A || !out) return -1;
  uint64_t total = (n >= 65) ? 0 : (1ull << (n - 1));
  if (first > total || count > total - first) return -1;
  int x[ORACLE_NMAX + 2];
  ld wr[ORACLE_NMAX], wi[ORACLE_NMAX];
  /* step 2: x := xor(r, rshift(r)) */
  unrank(first, n, x);
  /* step 3: t := (-1)^r */
  int t = (first & 1) ? -1 : 1;
  /* step 4: S := 0 */
  csum sr = {0, 0}, si = {0, 0}, sa = {0, 0};
  /* step 5: w_i := a_{i,n} - 1/2 sum_j a_{i,j} */
  for (int i = 0; i < n; ++i) {
    ld rr = 0, ri = 0;
    for (int j = 0; j < n; ++j) rr += RE(A, n, i, j), ri += IM(A, n, i, j);
    const int jn = MUT(3) ? 0 : n - 1;
    const ld half = MUT(5) ? 1 : 2;
    wr[i] = RE(A, n, i, jn) - rr / half;
    wi[i] = IM(A, n, i, jn) - ri / half;
  }
  /* steps 6-8: add the columns j < n whose bit x_j is set */
  for (int j = 1; j <= n - 1; ++j)
    if (x[j])
      for (int i = 0; i < n; ++i) wr[i] += RE(A, n, i, j - 1), wi[i] += IM(A, n, i, j - 1);
  /* steps 9-15 */
  for (uint64_t step = 0; step < count; ++step) {
    ld pr = 1, pi = 0; /* step 10: p := prod_i w_i */
    for (int i = 0; i < n - (MUT(1) ? 1 : 0); ++i) {
      ld nr = pr * wr[i] - pi * wi[i], ni = pr * wi[i] + pi * wr[i];
      pr = nr, pi = ni;
    }
    int j = nextset(&t, x, n); /* step 11 */
    csum_add(&sr, t * pr);     /* step 12: S := S + t p */
    csum_add(&si, t * pi);
    if (abs_sum) csum_add(&sa, sqrtl(pr * pr + pi * pi));
    int z = 2 * x[j] - 1; /* step 13 */
    for (int i = 0; i < n; ++i) { /* step 14: w_i := w_i + z a_{i,j} */
      const int ri_ = MUT(4) ? j - 1 : i, cj_ = MUT(4) ? i : j - 1;
      wr[i] += z * RE(A, n, ri_, cj_), wi[i] += z * IM(A, n, ri_, cj_);
    }
  }
  out[0] = csum_value(&sr);
  out[1] = csum_value(&si);
  if (abs_sum) *abs_sum = csum_value(&sa);
  return 0;
}

/* App. A "subpermanent(A, n, m, k, S)": part k of m. */
int oracle_glynn_part_c(const double* A, int n, uint64_t m, uint64_t k, ld* out, ld* abs_sum) {
  if (n < 1 || n > ORACLE_NMAX || m < 1 || k >= m) return -1;
  uint64_t r, l;
  distribute(1ull << (n - 1), m, k, &r, &l); /* step 1 */
  return oracle_glynn_range_c(A, n, r, l, out, abs_sum);
}

/* App. A "permanent(A, n, m, S)": S = 2 (-1)^n sum_k S_k.  The partials are
 * stored in an array and added in index order with compensation, as Sec. 2.B
 * advises instead of a plain reduction.  `threads` <= 0 uses the OpenMP
 * default. */
int oracle_per_glynn_c(const double* A, int n, int m, int threads, ld* out, ld* abs_sum) {
  if (n < 1 || n > ORACLE_NMAX || m < 1 || !A || !out) return -1;
  uint64_t total = 1ull << (n - 1);
  if ((uint64_t)m > total) m = (int)total;
  ld* part = (ld*)calloc((size_t)m * 3, sizeof(ld));
  if (!part) return -2;
  int err = 0;
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads) reduction(| : err)
#endif
  for (int k = 0; k < m; ++k) err |= oracle_glynn_part_c(A, n, (uint64_t)m, (uint64_t)k, &part[3 * k], &part[3 * k + 2]);
  csum sr = {0, 0}, si = {0, 0}, sa = {0, 0};
  for (int k = 0; k < m; ++k) {
    csum_add(&sr, part[3 * k]);
    csum_add(&si, part[3 * k + 1]);
    csum_add(&sa, part[3 * k + 2]);
  }
  free(part);
  ld s = ((n & 1) != MUT(6)) ? -2 : 2;
  out[0] = s * csum_value(&sr);
  out[1] = s * csum_value(&si);
  if (abs_sum) *abs_sum = 2 * csum_value(&sa);
  return err ? -1 : 0;
}

/* ======================================================================
 * Exact integer form.  With w_i as in App. A step 5, v_i = 2 w_i is an
 * integer for integer A:  v_i = 2 a_{i,n} - sum_j a_ij + 2 sum_{j<n, x_j=1} a_ij.
 * Then per(A) = 2 (-1)^n sum_r t_r prod_i w_i = 2^{1-n} (-1)^n sum_r t_r prod_i v_i.
 * The sum is carried in 512-bit two's-complement integers (8 x 64-bit limbs,
 * little endian), wide enough for |v_i| <= n*127 at n <= 36.
 * ==================================================================== */
#define XL 8
typedef struct {
  uint64_t l[XL];
} xint;

static void xint_set_i64(xint* a, int64_t v) {
  uint64_t fill = v < 0 ? ~0ull : 0ull;
  a->l[0] = (uint64_t)v;
  for (int i = 1; i < XL; ++i) a->l[i] = fill;
}

static void xint_add(xint* a, const xint* b) {
  unsigned __int128 carry = 0;
  for (int i = 0; i < XL; ++i) {
    unsigned __int128 s = (unsigned __int128)a->l[i] + b->l[i] + carry;
    a->l[i] = (uint64_t)s;
    carry = s >> 64;
  }
}

static void xint_neg(xint* a) {
  for (int i = 0; i < XL; ++i) a->l[i] = ~a->l[i];
  xint one;
  xint_set_i64(&one, 1);
  xint_add(a, &one);
}

static int xint_is_neg(const xint* a) { return (int)(a->l[XL - 1] >> 63); }

/* a := a * m for a signed 64-bit m (schoolbook on the magnitude) */
static void xint_mul_i64(xint* a, int64_t m) {
  int neg = 0;
  if (xint_is_neg(a)) xint_neg(a), neg ^= 1;
  uint64_t um = (uint64_t)m;
  if (m < 0) um = (uint64_t)0 - um, neg ^= 1;
  unsigned __int128 carry = 0;
  for (int i = 0; i < XL; ++i) {
    unsigned __int128 p = (unsigned __int128)a->l[i] * um + carry;
    a->l[i] = (uint64_t)p;
    carry = p >> 64;
  }
  if (neg) xint_neg(a);
}

/* Sum over code indices [first, first+count) of t_r * prod_i v_i, exactly,
 * with the paper's sign t.  Walk and updates follow App. A steps 2-15 with
 * v = 2w, so the column update is v_i := v_i + 2 z a_{i,j}. */
int oracle_glynn_exact_range_i8(const int8_t* A, int n, uint64_t first, uint64_t count, uint64_t* out /* XL limbs */) {
  if (n < 1 || n > 40 || !A || !out) return -1;
  uint64_t total = 1ull << (n - 1);
  if (first > total || count > total - first) return -1;
  /* overflow guard: 2^(n-1) * prod_i sum_j |a_ij| must stay below 2^(64*XL - 1) */
  double bits = (double)(n - 1);
  for (int i = 0; i < n; ++i) {
    int rs = 0;
    for (int j = 0; j < n; ++j) rs += abs((int)A[i * n + j]);
    if (rs == 0) rs = 1;
    bits += log2((double)rs) + 1e-9;
  }
  if (bits >= 64.0 * XL - 2) return -3;
  int x[ORACLE_NMAX + 2];
  int64_t v[ORACLE_NMAX];
  unrank(first, n, x);
  int t = (first & 1) ? -1 : 1;
  xint S;
  xint_set_i64(&S, 0);
  for (int i = 0; i < n; ++i) {
    int64_t rs = 0;
    for (int j = 0; j < n; ++j) rs += A[i * n + j];
    v[i] = 2 * (int64_t)A[i * n + n - 1] - rs;
  }
  for (int j = 1; j <= n - 1; ++j)
    if (x[j])
      for (int i = 0; i < n; ++i) v[i] += 2 * (int64_t)A[i * n + j - 1];
  for (uint64_t step = 0; step < count; ++step) {
    xint p;
    xint_set_i64(&p, 1);
    for (int i = 0; i < n; ++i) xint_mul_i64(&p, v[i]);
    int j = nextset(&t, x, n);
    if (t < 0) xint_neg(&p);
    xint_add(&S, &p);
    int z = 2 * x[j] - 1;
    for (int i = 0; i < n; ++i) v[i] += 2 * z * (int64_t)A[i * n + j - 1];
  }
  memcpy(out, S.l, sizeof(S.l));
  return 0;
}

/* Exact permanent of an integer matrix: 2^{1-n} (-1)^n times the full sum.
 * Returns -4 if the low n-1 bits are not zero (they must be). */
int oracle_per_exact_i8(const int8_t* A, int n, int m, int threads, uint64_t* out /* XL limbs */) {
  if (n < 1 || n > 40 || m < 1 || !A || !out) return -1;
  uint64_t total = 1ull << (n - 1);
  if ((uint64_t)m > total) m = (int)total;
  uint64_t* part = (uint64_t*)calloc((size_t)m * XL, sizeof(uint64_t));
  if (!part) return -2;
  int err = 0;
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads) reduction(| : err)
#endif
  for (int k = 0; k < m; ++k) {
    uint64_t r, l;
    distribute(total, (uint64_t)m, (uint64_t)k, &r, &l);
    int e = oracle_glynn_exact_range_i8(A, n, r, l, &part[(size_t)k * XL]);
    if (e) err |= 1;
  }
  xint S;
  xint_set_i64(&S, 0);
  for (int k = 0; k < m; ++k) {
    xint p;
    memcpy(p.l, &part[(size_t)k * XL], sizeof(p.l));
    xint_add(&S, &p);
  }
  free(part);
  if (err) return -1;
  /* times 2 (-1)^n, then divide by 2^n: overall 2^{1-n} (-1)^n */
  if (n & 1) xint_neg(&S);
  int neg = xint_is_neg(&S);
  if (neg) xint_neg(&S);
  int sh = n - 1; /* n - 1 < 64 */
  if (sh > 0) {
    if (S.l[0] & ((1ull << sh) - 1)) return -4;
    for (int i = 0; i < XL; ++i) {
      uint64_t hi = (i + 1 < XL) ? S.l[i + 1] : 0;
      S.l[i] = (S.l[i] >> sh) | (hi << (64 - sh));
    }
  }
  if (neg) xint_neg(&S);
  memcpy(out, S.l, sizeof(S.l));
  return 0;
}

/* ---- Modular form: the same sum of t_r prod_i v_i, reduced modulo each of k
 * odd moduli below 2^63.  Products use unsigned __int128 remainders. ---- */
static uint64_t mod_of_i64(int64_t v, uint64_t p) {
  int64_t r = v % (int64_t)p;
  if (r < 0) r += (int64_t)p;
  return (uint64_t)r;
}

int oracle_glynn_mod_range_i8(const int8_t* A, int n, const uint64_t* primes, int k, uint64_t first, uint64_t count,
                              uint64_t* out /* k */) {
  if (n < 1 || n > ORACLE_NMAX || !A || !primes || !out || k < 1 || k > 8) return -1;
  uint64_t total = 1ull << (n - 1);
  if (first > total || count > total - first) return -1;
  for (int q = 0; q < k; ++q)
    if (primes[q] < 3 || !(primes[q] & 1) || primes[q] >= (1ull << 63)) return -1;
  int x[ORACLE_NMAX + 2];
  int64_t v[ORACLE_NMAX];
  unrank(first, n, x);
  int t = (first & 1) ? -1 : 1;
  uint64_t S[8] = {0};
  for (int i = 0; i < n; ++i) {
    int64_t rs = 0;
    for (int j = 0; j < n; ++j) rs += A[i * n + j];
    v[i] = 2 * (int64_t)A[i * n + n - 1] - rs;
  }
  for (int j = 1; j <= n - 1; ++j)
    if (x[j])
      for (int i = 0; i < n; ++i) v[i] += 2 * (int64_t)A[i * n + j - 1];
  for (uint64_t step = 0; step < count; ++step) {
    int j = nextset(&t, x, n);
    for (int q = 0; q < k; ++q) {
      uint64_t p = primes[q];
      uint64_t prod = 1 % p;
      for (int i = 0; i < n; ++i) prod = (uint64_t)(((unsigned __int128)prod * mod_of_i64(v[i], p)) % p);
      if (t < 0 && prod) prod = p - prod;
      S[q] = (uint64_t)(((unsigned __int128)S[q] + prod) % p);
    }
    int z = 2 * x[j] - 1;
    for (int i = 0; i < n; ++i) v[i] += 2 * z * (int64_t)A[i * n + j - 1];
  }
  for (int q = 0; q < k; ++q) out[q] = S[q];
  return 0;
}

/* per(A) mod p_q for each modulus: 2^{1-n} (-1)^n sum_r t_r prod_i v_i (mod p). */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)(((unsigned __int128)a * b) % p); }

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = mulmod(r, a, p);
    a = mulmod(a, a, p);
    e >>= 1;
  }
  return r;
}

int oracle_per_mod_i8(const int8_t* A, int n, const uint64_t* primes, int k, int m, int threads, uint64_t* out) {
  if (n < 1 || n > ORACLE_NMAX || m < 1 || k < 1 || k > 8 || !A || !primes || !out) return -1;
  uint64_t total = 1ull << (n - 1);
  if ((uint64_t)m > total) m = (int)total;
  uint64_t* part = (uint64_t*)calloc((size_t)m * k, sizeof(uint64_t));
  if (!part) return -2;
  int err = 0;
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads) reduction(| : err)
#endif
  for (int c = 0; c < m; ++c) {
    uint64_t r, l;
    distribute(total, (uint64_t)m, (uint64_t)c, &r, &l);
    if (oracle_glynn_mod_range_i8(A, n, primes, k, r, l, &part[(size_t)c * k])) err |= 1;
  }
  for (int q = 0; q < k; ++q) {
    uint64_t p = primes[q], s = 0;
    for (int c = 0; c < m; ++c) s = (uint64_t)(((unsigned __int128)s + part[(size_t)c * k + q]) % p);
    /* times 2 (-1)^n / 2^n = (-1)^n / 2^(n-1); 2 is invertible mod odd p */
    uint64_t inv2 = (p + 1) / 2;
    s = mulmod(s, powmod(inv2, (uint64_t)(n - 1), p), p);
    if ((n & 1) && s) s = p - s;
    out[q] = s;
  }
  free(part);
  return err ? -1 : 0;
}

/* ---- Eq.(ryser2): A has R distinct columns cbar_1..cbar_R, column k
 * repeated m_k times (sum m_k = n).  C holds the distinct columns as an
 * n x R row-major complex array (C[i][k] = cbar_k(i)).
 *   per(A) = (-1)^n sum_{0 <= f_k <= m_k} (-1)^{sum f} (prod_k binom(m_k, f_k))
 *            prod_i sum_k f_k cbar_k(i)
 * The vectors f are visited in plain counting order (f_1 fastest); every
 * row sum is formed from scratch. */
static ld binom_ld(int m, int f) {
  ld b = 1;
  for (int t = 1; t <= f; ++t) b = b * (m - f + t) / t;
  return b;
}

int oracle_ryser2_c(const double* C, int n, int R, const int* mult, ld* out, ld* abs_sum) {
  if (n < 1 || n > ORACLE_NMAX || R < 1 || R > n || !C || !mult || !out) return -1;
  int tot = 0;
  for (int k = 0; k < R; ++k) {
    if (mult[k] < 1) return -1;
    tot += mult[k];
  }
  if (tot != n) return -1;
  int f[ORACLE_NMAX];
  for (int k = 0; k < R; ++k) f[k] = 0;
  csum sr = {0, 0}, si = {0, 0}, sa = {0, 0};
  for (;;) {
    ld wgt = 1;
    int fs = 0;
    for (int k = 0; k < R; ++k) wgt *= binom_ld(mult[k], f[k]), fs += f[k];
    ld pr = 1, pi = 0;
    for (int i = 0; i < n; ++i) {
      ld rr = 0, ri = 0;
      for (int k = 0; k < R; ++k) {
        rr += f[k] * (ld)C[2 * ((size_t)i * R + k)];
        ri += f[k] * (ld)C[2 * ((size_t)i * R + k) + 1];
      }
      ld nr = pr * rr - pi * ri, ni = pr * ri + pi * rr;
      pr = nr, pi = ni;
    }
    ld sg = (fs & 1) ? -wgt : wgt;
    csum_add(&sr, sg * pr);
    csum_add(&si, sg * pi);
    csum_add(&sa, wgt * sqrtl(pr * pr + pi * pi));
    /* next f in counting order */
    int k = 0;
    while (k < R && f[k] == mult[k]) f[k] = 0, ++k;
    if (k == R) break;
    ++f[k];
  }
  ld s = (n & 1) ? -1 : 1;
  out[0] = s * csum_value(&sr);
  out[1] = s * csum_value(&si);
  if (abs_sum) *abs_sum = csum_value(&sa);
  return 0;
}

/* ---- App. B "sparsepermanent(A, D, p)".  block[j] = l (0-based block index
 * of column j) for j in some S_l, or -1 for j in T.  The nested loops of the
 * listing ("for all non-empty s_l in S_l ... for all t in T") are run as one
 * mixed-radix counter whose digits are the bitmasks of s_1..s_d (1 .. 2^|S_l|-1)
 * and of t (0 .. 2^|T|-1). */
int oracle_sparse_c(const double* A, int n, const int* block, ld* out, ld* abs_sum) {
  if (n < 1 || n > 40 || !A || !block || !out) return -1;
  int d = 0;
  for (int j = 0; j < n; ++j) {
    if (block[j] < -1) return -1;
    if (block[j] + 1 > d) d = block[j] + 1;
  }
  /* column lists: digit 0..d-1 = blocks, digit d = T */
  int cols[ORACLE_NMAX + 1][ORACLE_NMAX], ncol[ORACLE_NMAX + 1];
  for (int l = 0; l <= d; ++l) ncol[l] = 0;
  for (int j = 0; j < n; ++j) {
    const int l = block[j] < 0 ? d : block[j];
    cols[l][ncol[l]++] = j;
  }
  for (int l = 0; l < d; ++l)
    if (ncol[l] == 0) return -1; /* every S_l is non-empty */
  uint64_t sub[ORACLE_NMAX + 1];
  for (int l = 0; l < d; ++l) sub[l] = 1; /* smallest non-empty subset */
  sub[d] = 0;
  csum sr = {0, 0}, si = {0, 0}, sa = {0, 0};
  for (;;) {
    /* J = s_1 u ... u s_d u t */
    int inJ[ORACLE_NMAX] = {0}, size = 0;
    for (int l = 0; l <= d; ++l)
      for (int b = 0; b < ncol[l]; ++b)
        if ((sub[l] >> b) & 1) inJ[cols[l][b]] = 1, ++size;
    ld pr = 1, pi = 0;
    for (int i = 0; i < n; ++i) {
      ld rr = 0, ri = 0;
      for (int j = 0; j < n; ++j)
        if (inJ[j]) rr += RE(A, n, i, j), ri += IM(A, n, i, j);
      ld nr = pr * rr - pi * ri, ni = pr * ri + pi * rr;
      pr = nr, pi = ni;
    }
    const ld sg = (size & 1) ? -1 : 1;
    csum_add(&sr, sg * pr);
    csum_add(&si, sg * pi);
    csum_add(&sa, sqrtl(pr * pr + pi * pi));
    /* next combination */
    int l = 0;
    for (; l <= d; ++l) {
      const uint64_t top = (1ull << ncol[l]) - 1;
      if (sub[l] < top) {
        ++sub[l];
        break;
      }
      sub[l] = l < d ? 1 : 0;
    }
    if (l > d) break;
  }
  const ld s = (n & 1) ? -1 : 1;
  out[0] = s * csum_value(&sr);
  out[1] = s * csum_value(&si);
  if (abs_sum) *abs_sum = csum_value(&sa);
  return 0;
}

int oracle_long_double_digits(void) { return LDBL_MANT_DIG; }

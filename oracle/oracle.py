"""ORACLE -- test infrastructure only.

Plain CPU reference for the permanent of Lundow & Markstrom (arXiv:1904.06229).
Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this module.  It shares no code with the CUDA library in the
package and never imports it.

What lives here:
  * ctypes bindings to `perm_oracle.c` (compiled on first use with gcc):
      - Eq.(per) brute force and Eq.(ryser) plain subset sum, long double;
      - App. A subpermanent / permanent (Gray-code walk, Neumaier-compensated
        long double accumulation, OpenMP over parts, fixed-order sum of parts);
      - exact 512-bit integer and multi-prime modular forms for int8 matrices.
  * pure-Python exact arithmetic for tiny cases:
      - Eq.(per) over all permutations with `fractions.Fraction`;
      - one Gray-code term evaluated straight from its definition (no walk);
      - Miller-Rabin primality and the four largest primes below 2^62;
      - Chinese remaindering with Python integers.

Sign and scaling conventions (App. A, "subpermanent" and "permanent"): the
term of code index r is prod_i w_i(x) with x = r xor (r >> 1) and
w_i = a_{i,n} - 1/2 sum_j a_ij + sum_{j<n, x_j=1} a_ij; the full permanent is
2 (-1)^(n-1) sum_r (-1)^r term(r).  `glynn_partial` returns
sum_{r in range} (-1)^r term(r) (the negative of the paper's S, whose sign t
is flipped before each addition).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from fractions import Fraction
from itertools import permutations

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "perm_oracle.c")
_SRC_PAPER = os.path.join(_HERE, "paper_scheme.c")  # the paper's double + Kahan CPU scheme (benchmark baseline)
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_XL = 8  # 64-bit limbs of the exact integer form
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile perm_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_PAPER))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, _SRC_PAPER]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            ld_p = ctypes.c_void_p
            u64 = ctypes.c_uint64
            lib.oracle_per_brute_c.argtypes = [ld_p, ctypes.c_int, ld_p]
            lib.oracle_per_ryser_c.argtypes = [ld_p, ctypes.c_int, ld_p]
            lib.oracle_glynn_range_c.argtypes = [ld_p, ctypes.c_int, u64, u64, ld_p, ld_p]
            lib.oracle_glynn_part_c.argtypes = [ld_p, ctypes.c_int, u64, u64, ld_p, ld_p]
            lib.oracle_per_glynn_c.argtypes = [ld_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ld_p, ld_p]
            lib.oracle_glynn_exact_range_i8.argtypes = [ld_p, ctypes.c_int, u64, u64, ld_p]
            lib.oracle_per_exact_i8.argtypes = [ld_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ld_p]
            lib.oracle_glynn_mod_range_i8.argtypes = [ld_p, ctypes.c_int, ld_p, ctypes.c_int, u64, u64, ld_p]
            lib.oracle_per_mod_i8.argtypes = [ld_p, ctypes.c_int, ld_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ld_p]
            lib.oracle_ryser2_c.argtypes = [ld_p, ctypes.c_int, ctypes.c_int, ld_p, ld_p, ld_p]
            lib.oracle_sparse_c.argtypes = [ld_p, ctypes.c_int, ld_p, ld_p, ld_p]
            lib.paper_scheme_range.argtypes = [ld_p, ctypes.c_int, u64, u64, ctypes.c_int, ctypes.c_int, ld_p]
            _lib = lib
    return _lib


def _as_c128(A) -> np.ndarray:
    """Row-major interleaved (re, im) float64 copy of a square matrix."""
    A = np.asarray(A)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    return np.ascontiguousarray(A.astype(np.complex128)).view(np.float64)


def _as_i8(A) -> np.ndarray:
    A = np.asarray(A)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    if np.any(np.abs(A.astype(np.int64)) > 127):
        raise ValueError("entries must fit int8")
    return np.ascontiguousarray(A.astype(np.int8))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _ld_complex(out: np.ndarray):
    return out[0], out[1]


def long_double_digits() -> int:
    return int(_load().oracle_long_double_digits())


# ----------------------------------------------------------------- long double
def per_brute(A):
    """Eq.(per) summed over all permutations in long double (n <= 10).

    Returns (re, im) as numpy longdouble."""
    a = _as_c128(A)
    out = np.zeros(2, dtype=np.longdouble)
    if _load().oracle_per_brute_c(_ptr(a), a.shape[0], _ptr(out)) != 0:
        raise ValueError("n out of range for brute force")
    return _ld_complex(out)


def per_ryser(A):
    """Eq.(ryser): plain inclusion-exclusion over all 2^n subsets (n <= 24)."""
    a = _as_c128(A)
    out = np.zeros(2, dtype=np.longdouble)
    if _load().oracle_per_ryser_c(_ptr(a), a.shape[0], _ptr(out)) != 0:
        raise ValueError("n out of range for Ryser")
    return _ld_complex(out)


def per(A, parts: int = 0, threads: int = 0):
    """App. A "permanent": Gray-code Glynn walk in `parts` parts (default: one
    part per 2^16 codes, at least one per thread), compensated long double.

    Returns (re, im, abs_sum) as numpy longdouble, abs_sum = sum over terms of
    |2 * term| (so abs_sum / |per| is the condition number of the sum)."""
    a = _as_c128(A)
    n = a.shape[0]
    total = 1 << (n - 1)
    if parts <= 0:
        parts = max(min(total, 64), min(total >> 16, 1 << 20))
    out = np.zeros(2, dtype=np.longdouble)
    asum = np.zeros(1, dtype=np.longdouble)
    rc = _load().oracle_per_glynn_c(_ptr(a), n, int(parts), int(threads), _ptr(out), _ptr(asum))
    if rc != 0:
        raise ValueError(f"oracle_per_glynn_c failed ({rc})")
    return out[0], out[1], asum[0]


def glynn_partial(A, first: int, count: int):
    """sum_{r=first}^{first+count-1} (-1)^r prod_i w_i(gray(r)), by the App. A
    walk started at `first` (unrank + seed, steps 2-8) and run `count` steps.

    Returns (re, im, abs_sum) as numpy longdouble."""
    a = _as_c128(A)
    n = a.shape[0]
    out = np.zeros(2, dtype=np.longdouble)
    asum = np.zeros(1, dtype=np.longdouble)
    rc = _load().oracle_glynn_range_c(_ptr(a), n, int(first), int(count), _ptr(out), _ptr(asum))
    if rc != 0:
        raise ValueError("bad range")
    # the paper's S carries t = (-1)^(r+1); negate to (-1)^r
    return -out[0], -out[1], asum[0]


def glynn_partial_parts(A, first: int, count: int, parts: int, threads: int = 0):
    """Same sum as `glynn_partial`, split into `parts` sub-ranges by the paper's
    `distribute`, evaluated in a thread pool of OpenMP-free ctypes calls and
    added in index order with compensation (long double)."""
    from concurrent.futures import ThreadPoolExecutor

    parts = max(1, min(parts, count)) if count else 1
    q, rem = divmod(count, parts)
    ranges = [(first + i * q + min(i, rem), q + (1 if i < rem else 0)) for i in range(parts)]
    workers = threads if threads > 0 else (os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=workers) as ex:
        res = list(ex.map(lambda fr: glynn_partial(A, fr[0], fr[1]), ranges))
    return _compensated([r[0] for r in res]), _compensated([r[1] for r in res]), _compensated([r[2] for r in res])


def paper_scheme_partial(A, first: int, count: int, parts: int, threads: int = 0):
    """The paper's CPU scheme (Sec. 2.B: double row sums and products, Kahan
    summation, consecutive parts in parallel, partials added in order) over
    the code range [first, first + count): sum (-1)^r prod_i w_i as a
    complex.  A benchmark baseline, not a parity reference."""
    a = _as_c128(A)
    out = np.zeros(2, dtype=np.float64)
    rc = _load().paper_scheme_range(_ptr(a), a.shape[0], int(first), int(count), int(parts), int(threads),
                                    _ptr(out))
    if rc != 0:
        raise ValueError("bad range")
    return complex(out[0], out[1])


def _compensated(xs):
    s = np.longdouble(0)
    c = np.longdouble(0)
    for x in xs:
        x = np.longdouble(x)
        t = s + x
        if abs(s) >= abs(x):
            c += (s - t) + x
        else:
            c += (x - t) + s
        s = t
    return s + c


def per_repeated(Cbar, mult):
    """Eq.(ryser2): permanent of the n x n matrix whose distinct columns are the
    R columns of `Cbar` (n x R), column k repeated mult[k] times.  Long double,
    plain counting order over the multiplicity vectors.  Returns (re, im,
    abs_sum), abs_sum = the sum of the terms' magnitudes (for error bounds)."""
    c = np.ascontiguousarray(np.asarray(Cbar).astype(np.complex128)).view(np.float64)
    Cb = np.asarray(Cbar)
    n, R = Cb.shape
    m = np.ascontiguousarray(np.asarray(mult, dtype=np.int32))
    out = np.zeros(2, dtype=np.longdouble)
    asum = np.zeros(1, dtype=np.longdouble)
    rc = _load().oracle_ryser2_c(_ptr(c), int(n), int(R), _ptr(m), _ptr(out), _ptr(asum))
    if rc != 0:
        raise ValueError("bad repeated-column specification")
    return out[0], out[1], asum[0]


# ------------------------------------------------------------------- integers
def _limbs_to_int(limbs) -> int:
    v = 0
    for i, l in enumerate(limbs):
        v |= int(l) << (64 * i)
    if v >> (64 * _XL - 1):
        v -= 1 << (64 * _XL)
    return v


def per_exact(A, parts: int = 0, threads: int = 0) -> int:
    """Exact permanent of an integer (int8) matrix via the integer form of the
    App. A walk (v = 2w), 512-bit accumulation, exact division by 2^(n-1)."""
    a = _as_i8(A)
    n = a.shape[0]
    if parts <= 0:
        parts = max(1, min(1 << (n - 1), 4096))
    out = np.zeros(_XL, dtype=np.uint64)
    rc = _load().oracle_per_exact_i8(_ptr(a), n, int(parts), int(threads), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_per_exact_i8 failed ({rc})")
    return _limbs_to_int(out)


def glynn_exact_partial(A, first: int, count: int) -> int:
    """Exact sum_{r in range} (-1)^r prod_i v_i(gray(r)) with v = 2w (integer A)."""
    a = _as_i8(A)
    out = np.zeros(_XL, dtype=np.uint64)
    rc = _load().oracle_glynn_exact_range_i8(_ptr(a), a.shape[0], int(first), int(count), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_glynn_exact_range_i8 failed ({rc})")
    return -_limbs_to_int(out)


def per_mod(A, primes, parts: int = 0, threads: int = 0):
    """per(A) mod each prime, by the modular form of the walk (int8 A)."""
    a = _as_i8(A)
    n = a.shape[0]
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64))
    if parts <= 0:
        parts = max(1, min(1 << (n - 1), 4096))
    out = np.zeros(len(pr), dtype=np.uint64)
    rc = _load().oracle_per_mod_i8(_ptr(a), n, _ptr(pr), len(pr), int(parts), int(threads), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_per_mod_i8 failed ({rc})")
    return [int(v) for v in out]


# ------------------------------------------------------ exact tiny references
def _frac(x) -> Fraction:
    return Fraction(float(x))


def per_brute_exact(A):
    """Eq.(per) over all n! permutations, exact rational arithmetic.

    Float entries are taken at their exact binary values.  Returns a pair of
    Fractions (re, im)."""
    A = np.asarray(A)
    n = A.shape[0]
    if n > 8:
        raise ValueError("n <= 8 for the exact brute force")
    M = [[(_frac(np.real(A[i, j])), _frac(np.imag(A[i, j]))) for j in range(n)] for i in range(n)]
    sr, si = Fraction(0), Fraction(0)
    for p in permutations(range(n)):
        pr, pi = Fraction(1), Fraction(0)
        for i in range(n):
            ar, ai = M[i][p[i]]
            pr, pi = pr * ar - pi * ai, pr * ai + pi * ar
        sr += pr
        si += pi
    return sr, si


def per_brute_int(A) -> int:
    """Eq.(per) over all n! permutations for integer A (Python integers)."""
    A = np.asarray(A, dtype=np.int64)
    n = A.shape[0]
    s = 0
    for p in permutations(range(n)):
        t = 1
        for i in range(n):
            t *= int(A[i, p[i]])
        s += t
    return s


def glynn_term_exact(A, r: int):
    """One term of the halved Gray-code sum, straight from its definition:
    (-1)^r prod_i (a_{i,n} - 1/2 sum_j a_ij + sum_{j<n: x_j=1} a_ij),
    x = r xor (r >> 1); exact rational (re, im)."""
    A = np.asarray(A)
    n = A.shape[0]
    x = r ^ (r >> 1)
    M = [[(_frac(np.real(A[i, j])), _frac(np.imag(A[i, j]))) for j in range(n)] for i in range(n)]
    pr, pi = Fraction(1), Fraction(0)
    for i in range(n):
        wr = M[i][n - 1][0] - sum(M[i][j][0] for j in range(n)) / 2
        wi = M[i][n - 1][1] - sum(M[i][j][1] for j in range(n)) / 2
        for j in range(n - 1):
            if (x >> j) & 1:
                wr += M[i][j][0]
                wi += M[i][j][1]
        pr, pi = pr * wr - pi * wi, pr * wi + pi * wr
    s = -1 if r & 1 else 1
    return s * pr, s * pi


def band_permanent_exact(A, k: int):
    """App. C "bandpermanent(A, k, p)" in exact rational arithmetic.

    The polynomial p in the formal variables x_1..x_n is a dict from the
    bitmask of a multilinear monomial to its coefficient (a pair of
    Fractions).  For each row i: p := p * C_i with C_i = sum_j a_ij x_j
    (only the entries inside the band |i - j| <= k; x_j^2 = 0 drops products
    that repeat a variable), then x_{i-k-1} := 1 (its bit is cleared, merging
    monomials); finally every x := 1 (the coefficients are summed).  The
    entries outside the band must be zero (checked)."""
    A = np.asarray(A)
    n = A.shape[0]
    for i in range(n):
        for j in range(n):
            if abs(i - j) > k and A[i, j] != 0:
                raise ValueError("entry outside the band")
    M = [[(_frac(np.real(A[i, j])), _frac(np.imag(A[i, j]))) for j in range(n)] for i in range(n)]
    p = {0: (Fraction(1), Fraction(0))}
    for i in range(n):  # 0-based row i is the paper's row i+1
        q = {}
        for S, (cr, ci) in p.items():
            for j in range(max(0, i - k), min(n, i + k + 1)):
                if (S >> j) & 1:
                    continue  # x_j^2 = 0
                ar, ai = M[i][j]
                if ar == 0 and ai == 0:
                    continue
                T = S | (1 << j)
                tr, ti = q.get(T, (Fraction(0), Fraction(0)))
                q[T] = (tr + cr * ar - ci * ai, ti + cr * ai + ci * ar)
        r = i - k - 1  # 0-based index of x_{i-k-1} for the paper's row i+1
        if r >= 0:
            merged = {}
            for S, (cr, ci) in q.items():
                S2 = S & ~(1 << r)
                tr, ti = merged.get(S2, (Fraction(0), Fraction(0)))
                merged[S2] = (tr + cr, ti + ci)
            q = merged
        p = q
    sr = sum((c[0] for c in p.values()), Fraction(0))
    si = sum((c[1] for c in p.values()), Fraction(0))
    return sr, si


def greedy_partition(A, rng=None):
    """App. B "greedypartition(A, D)": b_ij = [a_ij != 0]; repeatedly take a
    row k of least out-degree among the rows left in V (ties: the first, or a
    random one when `rng` is given), make S_d = N_k (the columns of its
    non-zeros), remove k and every row whose neighbourhood meets N_k from V;
    T = the columns in no S_l.  Returns block[j] = l for j in S_l, -1 for T."""
    A = np.asarray(A)
    n = A.shape[0]
    b = (A != 0)
    deg = b.sum(axis=1)
    nbr = [set(np.nonzero(b[i])[0].tolist()) for i in range(n)]
    V = set(range(n))
    blocks = []
    while V:
        dmin = min(deg[i] for i in V)
        cands = sorted(i for i in V if deg[i] == dmin)
        k = cands[0] if rng is None else cands[int(rng.integers(len(cands)))]
        Nk = nbr[k]
        blocks.append(sorted(Nk))
        V.discard(k)
        for l in list(V):
            if Nk & nbr[l]:
                V.discard(l)
    block = [-1] * n
    for l, S in enumerate(blocks):
        for j in S:
            block[j] = l
    return block


def partition_count(block) -> int:
    """Number of sets the restricted sum visits: 2^|T| prod_l (2^|S_l| - 1)."""
    from collections import Counter

    c = Counter(block)
    tot = 1 << c.get(-1, 0)
    for l, s in c.items():
        if l >= 0:
            tot *= (1 << s) - 1
    return tot


def per_sparse(A, block=None):
    """App. B "sparsepermanent" with the partition `block` (default: the
    deterministic greedy partition).  Returns (re, im, abs_sum), long double."""
    a = _as_c128(A)
    n = a.shape[0]
    if block is None:
        block = greedy_partition(A)
    bl = np.ascontiguousarray(np.asarray(block, dtype=np.int32))
    out = np.zeros(2, dtype=np.longdouble)
    asum = np.zeros(1, dtype=np.longdouble)
    rc = _load().oracle_sparse_c(_ptr(a), n, _ptr(bl), _ptr(out), _ptr(asum))
    if rc != 0:
        raise ValueError("bad sparse partition")
    return out[0], out[1], asum[0]


STATS_STRIDE = 103


def batch_stats(pers, ns):
    """Statistics of X = |per| / sqrt(n!) per order n = 0..32 (Secs. 3-6):
    row n = [count, sum X, sum X^2, sum X^3, sum X^4, histogram...] with 16
    bins per decade: bin 0 for X < 1e-4, bin b = 1..96 for
    10^(-4+(b-1)/16) <= X < 10^(-4+b/16), bin 97 for X >= 100.  Sums are
    exactly rounded (math.fsum)."""
    edges = [10.0 ** (-4.0 + j / 16.0) for j in range(97)]
    out = np.zeros((33, STATS_STRIDE))
    xs = {}
    for p, n in zip(pers, ns):
        x = abs(complex(p)) / math.sqrt(math.factorial(int(n)))
        xs.setdefault(int(n), []).append(x)
    for n, v in xs.items():
        out[n, 0] = len(v)
        for q in range(1, 5):
            out[n, q] = math.fsum(x ** q for x in v)
        for x in v:
            b = sum(1 for e in edges if e <= x)
            out[n, 5 + b] += 1
    return out


# ------------------------------------------------------- primes and the CRT
def is_prime(m: int) -> bool:
    """Deterministic Miller-Rabin for m < 3.3e24 (first twelve prime bases)."""
    if m < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if m % p == 0:
            return m == p
    d, s = m - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        y = pow(a, d, m)
        if y in (1, m - 1):
            continue
        for _ in range(s - 1):
            y = y * y % m
            if y == m - 1:
                break
        else:
            return False
    return True


def largest_primes_below(bound: int, k: int):
    out = []
    c = bound - 1
    while len(out) < k:
        if is_prime(c):
            out.append(c)
        c -= 1
    return out


def default_primes():
    """The four largest primes below 2^62 (found by search, not typed in)."""
    return largest_primes_below(1 << 62, 4)


def crt(residues, primes) -> int:
    """Chinese remaindering; result centred in (-P/2, P/2]."""
    P = 1
    for p in primes:
        P *= p
    x = 0
    for r, p in zip(residues, primes):
        Mi = P // p
        x += int(r) * Mi * pow(Mi, -1, p)
    x %= P
    if x > P // 2:
        x -= P
    return x

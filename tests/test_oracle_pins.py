"""Pins for the CPU oracle: it is checked against what the paper and the
mathematics fix, never against itself or the CUDA library.

  * Eq.(per) brute force with exact rational arithmetic (n <= 8);
  * worked examples under tests/golden/ (hand-derived, cited);
  * closed forms: per(J_n) = n! (Sec. 2.B), per(I) = 1, permutation matrices,
    per(J - I) = derangement numbers, rank one, block diagonal;
  * invariances: row/column permutation, transpose, multilinearity;
  * the range form against single terms computed from their definition;
  * exact integer, modular and CRT forms against each other and brute force.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_06229_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _c(re, im=0):
    return complex(float(re), float(im))


def _ld_rel(got_re, got_im, ref_re, ref_im):
    d = np.hypot(np.longdouble(got_re) - np.longdouble(ref_re), np.longdouble(got_im) - np.longdouble(ref_im))
    m = np.hypot(np.longdouble(ref_re), np.longdouble(ref_im))
    return float(d / m) if m else float(d)


def _u_ld():
    return 2.0 ** (1 - O.long_double_digits())


def derangements(n):
    d = [1, 0]
    for k in range(2, n + 1):
        d.append((k - 1) * (d[k - 1] + d[k - 2]))
    return d[n]


@pytest.mark.parametrize("n", range(1, 9))
def test_brute_force_exact(n):
    A = W.complex_gaussian(n, 100 + n)
    er, ei = O.per_brute_exact(A)
    ref = (np.longdouble(er.numerator) / np.longdouble(er.denominator),
           np.longdouble(ei.numerator) / np.longdouble(ei.denominator))
    tol = 64 * n * _u_ld() * 50
    for f in (O.per_brute, O.per_ryser):
        r = f(A) if n <= 8 else None
        assert _ld_rel(r[0], r[1], *ref) < tol
    g = O.per(A)
    assert _ld_rel(g[0], g[1], *ref) < max(tol, 64 * n * _u_ld() * float(g[2] / np.hypot(*ref)))


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_golden_worked_examples(case):
    A = np.array(case["matrix"], dtype=float)
    r = O.per(A)
    assert float(r[0]) == pytest.approx(case["per"], rel=1e-15, abs=1e-15)
    assert abs(float(r[1])) < 1e-15
    if np.allclose(A, np.round(A)) and np.abs(A).max() < 128:
        assert O.per_exact(A.astype(np.int8)) == case["per"]
        assert O.per_brute_int(A.astype(np.int64)) == case["per"]


def test_hand_traces_small():
    # n = 1: per = a ; n = 2: per = ad + bc (App. A traced by hand)
    a, b, c, d = 1.25 - 0.5j, -2.0 + 0.75j, 0.5 + 3j, -1.5 - 1j
    r = O.per(np.array([[a]]))
    assert _c(r[0], r[1]) == a
    r = O.per(np.array([[a, b], [c, d]]))
    assert abs(_c(r[0], r[1]) - (a * d + b * c)) < 1e-15
    # n = 3: sum over the six permutations written out
    M = W.complex_gaussian(3, 7)
    p = (M[0, 0] * M[1, 1] * M[2, 2] + M[0, 0] * M[1, 2] * M[2, 1] + M[0, 1] * M[1, 0] * M[2, 2]
         + M[0, 1] * M[1, 2] * M[2, 0] + M[0, 2] * M[1, 0] * M[2, 1] + M[0, 2] * M[1, 1] * M[2, 0])
    r = O.per(M)
    assert abs(_c(r[0], r[1]) - p) < 1e-14 * abs(p)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 16, 20, 24])
def test_all_ones_factorial(n):
    # Sec. 2.B: per(J) = n!
    r = O.per(np.ones((n, n)))
    assert _ld_rel(r[0], r[1], math.factorial(n), 0) < 1e-14
    if n <= 20:
        assert O.per_exact(np.ones((n, n), dtype=np.int8)) == math.factorial(n)


@pytest.mark.parametrize("n", [1, 4, 9, 16])
def test_identity_and_permutation(n):
    r = O.per(np.eye(n))
    assert _c(r[0], r[1]) == 1
    P = np.eye(n)[np.random.default_rng(n).permutation(n)]
    r = O.per(P)
    assert abs(_c(r[0], r[1]) - 1) < 1e-15
    assert O.per_exact(P.astype(np.int8)) == 1


@pytest.mark.parametrize("n", [2, 3, 5, 8, 11, 14, 18])
def test_derangements(n):
    J = np.ones((n, n)) - np.eye(n)
    Dn = derangements(n)
    r = O.per(J)
    assert _ld_rel(r[0], r[1], Dn, 0) < 1e-14
    assert O.per_exact(J.astype(np.int8)) == Dn


@pytest.mark.parametrize("n", [3, 6, 10, 13])
def test_rank_one(n):
    rng = np.random.default_rng(50 + n)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = math.factorial(n) * np.prod(u) * np.prod(v)
    r = O.per(np.outer(u, v))
    tol = 256 * n * _u_ld() * float(r[2]) / abs(ref) + 1e-15
    assert abs(_c(r[0], r[1]) - ref) <= tol * abs(ref)


def test_block_diagonal():
    B = W.complex_gaussian(7, 1)
    C = W.haar_submatrix(6, 36, 2)
    M = np.zeros((13, 13), dtype=complex)
    M[:7, :7] = B
    M[7:, 7:] = C
    pb, pc, pm = O.per(B), O.per(C), O.per(M)
    ref = _c(pb[0], pb[1]) * _c(pc[0], pc[1])
    assert abs(_c(pm[0], pm[1]) - ref) < 1e-13 * abs(ref)


def test_invariances():
    n = 11
    A = W.complex_gaussian(n, 9)
    r0 = O.per(A)
    p0 = _c(r0[0], r0[1])
    rng = np.random.default_rng(0)
    for B in (A.T, A[rng.permutation(n)], A[:, rng.permutation(n)],
              A[rng.permutation(n)][:, rng.permutation(n)]):
        r = O.per(B)
        assert abs(_c(r[0], r[1]) - p0) < 1e-13 * abs(p0)
    # multilinearity in a row
    c = 0.75 - 2.5j
    B = A.copy()
    B[4] *= c
    r = O.per(B)
    assert abs(_c(r[0], r[1]) - c * p0) < 1e-13 * abs(c * p0)


@pytest.mark.parametrize("n", [9, 12, 14])
def test_ryser_vs_glynn(n):
    A = W.haar_submatrix(n, n * n, 11 + n)
    a, b = O.per_ryser(A), O.per(A)
    assert _ld_rel(b[0], b[1], a[0], a[1]) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_range_terms_from_definition(n):
    """Every single-code range equals the term computed from its definition."""
    A = W.complex_gaussian(n, 30 + n)
    for r in range(1 << (n - 1)):
        tr, ti = O.glynn_term_exact(A, r)
        g = O.glynn_partial(A, r, 1)
        ref = (float(tr), float(ti))
        assert abs(_c(g[0], g[1]) - complex(*ref)) <= 1e-15 * max(1.0, abs(complex(*ref)))


def test_range_partition_sums_to_permanent():
    n = 13
    A = W.complex_gaussian(n, 77)
    N = 1 << (n - 1)
    cuts = [0, 1, 7, 100, 1023, 1024, 3000, N - 1, N]
    re = im = np.longdouble(0)
    for a, b in zip(cuts[:-1], cuts[1:]):
        g = O.glynn_partial(A, a, b - a)
        re += g[0]
        im += g[1]
    s = 2 * (-1) ** (n - 1)
    r = O.per(A)
    assert _ld_rel(s * re, s * im, r[0], r[1]) < 1e-14
    g = O.glynn_partial_parts(A, 0, N, 5)
    assert _ld_rel(s * g[0], s * g[1], r[0], r[1]) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_exact_integer_vs_brute(n):
    rng = np.random.default_rng(200 + n)
    for A in (W.zero_one(n, n), W.bernoulli_pm1(n, n), rng.integers(-127, 128, (n, n))):
        assert O.per_exact(A) == O.per_brute_int(A)


def test_exact_integer_partial_divisibility():
    # the unscaled full sum is 2^(n-1) * per * (-1)^(n-1) / 2 ... checked through per_exact's own divisibility
    n = 10
    A = W.bernoulli_pm1(n, 3)
    N = 1 << (n - 1)
    tot = sum(O.glynn_exact_partial(A, a, b - a) for a, b in [(0, 5), (5, 300), (300, N)])
    # per = 2^(1-n) (-1)^(n-1) * sum_r (-1)^r prod v_r
    assert tot % (1 << (n - 1)) == 0
    assert (tot >> (n - 1)) * (-1) ** (n - 1) == O.per_exact(A)


def test_primes():
    ps = O.default_primes()
    assert len(ps) == 4 and len(set(ps)) == 4
    sympy = pytest.importorskip("sympy")
    for p in ps:
        assert p < 2**62 and p % 2 == 1 and sympy.isprime(p)
    # they are the four largest below 2^62
    assert ps[0] == sympy.prevprime(2**62)
    for a, b in zip(ps[:-1], ps[1:]):
        assert sympy.prevprime(a) == b


@pytest.mark.parametrize("n", [3, 9, 14])
def test_modular_and_crt(n):
    ps = O.default_primes()
    for A in (W.zero_one(n, 60 + n), W.bernoulli_pm1(n, 70 + n)):
        ex = O.per_exact(A)
        res = O.per_mod(A, ps)
        assert res == [ex % p for p in ps]
        assert O.crt(res, ps) == ex


def test_crt_signed_roundtrip():
    ps = O.default_primes()
    for v in (0, 1, -1, 3**100, -(7**80), (1 << 200) + 12345):
        assert O.crt([v % p for p in ps], ps) == v


def test_condition_number_reported():
    A = W.complex_gaussian(12, 5)
    r = O.per(A)
    assert r[2] >= np.hypot(r[0], r[1])


# ---------------------------------------------------------------- Eq.(ryser2)
@pytest.mark.parametrize("mult", [[1], [3], [2, 1], [1, 1, 1], [2, 2, 1], [4, 1, 2], [1, 3, 1, 2], [5, 5]])
def test_ryser2_vs_brute_on_expanded(mult):
    n = sum(mult)
    Cb = W.complex_gaussian(n, 90 + n)[:, :len(mult)]
    A = W.expand_columns(Cb, mult)
    r2 = O.per_repeated(Cb, mult)
    if n <= 8:
        er, ei = O.per_brute_exact(A)
        ref = (np.longdouble(er.numerator) / np.longdouble(er.denominator),
               np.longdouble(ei.numerator) / np.longdouble(ei.denominator))
    else:
        g = O.per(A)
        ref = (g[0], g[1])
    assert _ld_rel(r2[0], r2[1], *ref) < 1e-14


def test_ryser2_closed_forms():
    # one distinct column of ones repeated n times: per(J_n) = n!
    for n in (1, 4, 9, 15):
        r = O.per_repeated(np.ones((n, 1)), [n])
        assert _ld_rel(r[0], r[1], math.factorial(n), 0) < 1e-15
    # one column c repeated n times: per = n! prod_i c_i
    c = W.complex_gaussian(6, 3)[:, :1]
    r = O.per_repeated(c, [6])
    ref = math.factorial(6) * np.prod(c[:, 0])
    assert abs(complex(float(r[0]), float(r[1])) - ref) < 1e-13 * abs(ref)


# ------------------------------------------------------- App. C band-limited
@pytest.mark.parametrize("n,k", [(1, 0), (4, 0), (5, 1), (7, 2), (8, 3), (8, 7)])
def test_band_vs_brute(n, k):
    A = W.band_matrix(n, k, 10 * n + k)
    br, bi = O.band_permanent_exact(A, k)
    er, ei = O.per_brute_exact(A)
    assert (br, bi) == (er, ei)  # both exact rationals


@pytest.mark.parametrize("n,k", [(14, 1), (16, 2), (18, 3)])
def test_band_vs_glynn(n, k):
    A = W.band_matrix(n, k, 5 + n, kind="real" if k == 2 else "gaussian")
    br, bi = O.band_permanent_exact(A, k)
    g = O.per(A)
    ref = complex(float(g[0]), float(g[1]))
    assert abs(complex(float(br), float(bi)) - ref) <= 1e-13 * abs(ref)


def test_band_tridiagonal_fibonacci():
    # per of the n x n tridiagonal all-ones matrix is the Fibonacci number F_{n+1}
    fib = [0, 1]
    for _ in range(40):
        fib.append(fib[-1] + fib[-2])
    for n in (1, 2, 3, 10, 25):
        A = W.band_matrix(n, 1, 0) * 0
        i, j = np.indices((n, n))
        A[np.abs(i - j) <= 1] = 1
        br, bi = O.band_permanent_exact(A, 1)
        assert br == fib[n + 1] and bi == 0


# ------------------------------------------------- statistics of Secs. 3-6
def test_batch_stats_bins_and_sums():
    import math as _m
    pers = [1.0, _m.sqrt(2.0) * 1.0, 1e-6, 1e3, 10 ** (1 / 16) * 0.999999]
    ns = [1, 2, 1, 1, 1]
    st = O.batch_stats(pers, ns)
    assert st[1, 0] == 4 and st[2, 0] == 1
    assert st[:, 5:].sum() == 5
    assert st[1, 5 + 0] == 1          # 1e-6 below 1e-4
    assert st[1, 5 + 97] == 1         # 1e3 above 100
    assert st[1, 5 + 65] == 2         # X = 1 and X just below 10^(1/16): [10^0, 10^(1/16))
    assert st[2, 5 + 65] == 1         # |per| / sqrt(2!) = 1
    assert st[1, 2] == pytest.approx(1.0 + 1e-12 + 1e6 + (10 ** (1 / 16) * 0.999999) ** 2, rel=1e-15)


def test_batch_stats_second_moment_gaussian():
    # Sec. 3: <X^2> = 1 for independent variance-1 entries
    n, m = 6, 3000
    pers = []
    for k in range(m):
        r = O.per(W.complex_gaussian(n, 20_000 + k))
        pers.append(complex(float(r[0]), float(r[1])))
    st = O.batch_stats(pers, [n] * m)
    mean_x2 = st[n, 2] / st[n, 0]
    se = math.sqrt(n / m)  # <X^4> = n + 1 gives Var(X^2) = n
    assert abs(mean_x2 - 1.0) < 5 * se


# ------------------------------------------------------ App. B sparse matrices
@pytest.mark.parametrize("n,p,seed", [(6, 0.2, 1), (8, 0.1, 2), (12, 0.1, 3), (16, 0.05, 4), (18, 0.15, 5)])
def test_sparse_vs_glynn(n, p, seed):
    A = W.sparse_matrix(n, p, seed)
    block = O.greedy_partition(A)
    assert O.partition_count(block) <= 1 << n
    r = O.per_sparse(A, block)
    g = O.per(A)
    ref = complex(float(g[0]), float(g[1]))
    got = complex(float(r[0]), float(r[1]))
    assert abs(got - ref) <= 1e-13 * abs(ref) + 64 * n * _u_ld() * float(r[2])
    if n <= 8:
        er, ei = O.per_brute_exact(A)
        assert abs(got - complex(float(er), float(ei))) <= 1e-13 * abs(ref)


def test_sparse_partition_properties():
    A = W.sparse_matrix(30, 0.05, 9)
    rng = np.random.default_rng(0)
    for block in (O.greedy_partition(A), O.greedy_partition(A, rng)):
        nb = max(block) + 1
        # blocks are neighbourhoods of rows, pairwise disjoint by construction
        for l in range(nb):
            S = {j for j in range(30) if block[j] == l}
            assert any(S == set(np.nonzero(A[i])[0].tolist()) for i in range(30))
        assert O.partition_count(block) < 1 << 30


def test_sparse_identity_and_permutation():
    for n in (1, 5, 11):
        r = O.per_sparse(np.eye(n, dtype=complex))
        assert complex(float(r[0]), float(r[1])) == 1
    P = np.eye(9, dtype=complex)[np.random.default_rng(2).permutation(9)] * 2.0
    r = O.per_sparse(P)
    assert complex(float(r[0]), float(r[1])) == 2.0 ** 9

"""The paper's CPU scheme (oracle/paper_scheme.c: double row sums and
products, Kahan summation, parts in parallel; the benchmark's second CPU
baseline) against the long-double oracle and Eq.(per) brute force."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_06229_gb300 import workloads as W


@pytest.mark.parametrize("n,first,count,parts", [(1, 0, 1, 1), (5, 0, 16, 3), (9, 7, 200, 4), (14, 100, 5000, 7),
                                                 (16, 0, 1 << 15, 16)])
def test_agrees_with_oracle_walk(n, first, count, parts):
    A = W.complex_gaussian(n, 60 + n)
    re, im, asum = O.glynn_partial(A, first, count)
    ref = complex(float(re), float(im))
    got = O.paper_scheme_partial(A, first, count, parts)
    # double products and row sums: about (2n + 2) 2^-53 per term
    assert abs(got - ref) <= (2 * n + 2) * 2.0 ** -53 * float(asum) * 4, (got, ref)


@pytest.mark.parametrize("n", [2, 4, 7])
def test_full_sum_is_the_permanent(n):
    A = W.complex_gaussian(n, 80 + n)
    s = O.paper_scheme_partial(A, 0, 1 << (n - 1), 3)
    per = 2 * (-1) ** (n - 1) * s
    br, bi = O.per_brute_exact(A)
    ref = complex(float(br), float(bi))
    assert abs(per - ref) <= 1e-12 * abs(ref) * math.factorial(n)


def test_rejects_bad_ranges():
    A = W.complex_gaussian(4, 1)
    with pytest.raises(ValueError):
        O.paper_scheme_partial(A, 7, 2, 1)

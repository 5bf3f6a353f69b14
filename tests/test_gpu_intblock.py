"""Edge cases of the complex walks' row scaling and product arithmetic (the
default packed double-float walk and the exact fixed-point walk with its
integer block floating point): exponent bookkeeping across rows of very
different scale, row sums that are exactly zero at many codes, and integer
matrices whose permanent is known exactly."""
import numpy as np
import pytest
import torch

import _tolerance as T
from oracle import oracle as O
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = T.REL


@pytest.fixture(autouse=True, params=["pdf", "fixed"])
def rows(request, monkeypatch):
    monkeypatch.setenv("PERM_ROWS", request.param)
    return request.param


def gpu_c128(A):
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.complex128))).cuda()
    r = P.perm_c128(t).cpu().numpy()
    assert P.perm_last_status() == 0
    return complex(r[0], r[1])


@pytest.mark.parametrize("n", [10, 24, 30])
def test_rows_of_very_different_scale(n):
    """Row i scaled by 2^s_i with sum s_i = 0: per is unchanged, and since each
    row's fixed-point scale absorbs its 2^s_i exactly, so is every term the
    kernel forms; the result must be the same double, bit for bit."""
    A = W.complex_gaussian(n, 900 + n)
    rng = np.random.default_rng(n)
    s = rng.integers(-30, 31, size=n)
    s[-1] = -int(s[:-1].sum())
    B = A * np.ldexp(1.0, s)[:, None]
    assert gpu_c128(B) == gpu_c128(A)


@pytest.mark.parametrize("n", [9, 16, 23])
def test_integer_matrices_exact(n):
    """+-1, 0-1 and all-ones matrices as complex128: many row sums are exactly
    zero at many codes; the result equals the exact integer permanent."""
    for A in (W.bernoulli_pm1(n, 40 + n), W.zero_one(n, 50 + n), np.ones((n, n), dtype=np.int8)):
        ex = O.per_exact(A)
        got = gpu_c128(A.astype(np.float64))
        assert got.imag == 0.0
        print(f"integer matrix n={n}: rel err {abs(got.real - ex) / abs(ex) if ex else abs(got.real):.3e}")
        assert abs(got.real - ex) <= REL * abs(ex) if ex else got.real == 0.0


@pytest.mark.parametrize("n", [12, 18])
def test_complex_unit_entries(n, rows):
    """Entries in {1, -1, i, -i} against the long-double oracle and the
    transpose."""
    k = np.random.default_rng(70 + n).integers(0, 4, size=(n, n))
    A = (1j) ** k
    re, im, asum = O.per(A)
    ref = complex(float(re), float(im))
    u = T.unit(rows)
    T.check(gpu_c128(A), ref, float(asum), n, u, f"unit entries n={n}")
    T.check(gpu_c128(A.T), ref, float(asum), n, u, f"unit entries n={n}, transpose")


@pytest.mark.parametrize("n", [7, 20])
def test_rows_of_extreme_magnitude(n, rows):
    """Rows scaled by 1e+-300 (not powers of two) and by 2^+-1000: each row's
    own scale absorbs its magnitude, so the result matches the long-double
    oracle of the scaled matrix (its range reaches 1e+-4932) at the bar."""
    A = W.complex_gaussian(n, 950 + n)
    s = np.ones(n)
    s[0], s[1] = 1e300, 1e-300
    s[2], s[3] = 2.0 ** 1000, 2.0 ** -1000
    B = A * s[:, None]
    re, im, asum = O.per(B)
    ref = complex(float(re), float(im))
    T.check(gpu_c128(B), ref, float(asum), n, T.unit(rows), f"extreme rows n={n}")


@pytest.mark.parametrize("n", [6, 19])
def test_zero_row_and_column(n, rows):
    """A zero row makes every term zero: per = 0 exactly.  A zero column makes
    per = 0 by cancellation of term pairs (codes that differ in that column),
    which the walk reaches to within the rounding of those terms: the
    a-posteriori bound with the oracle's sum of term magnitudes."""
    A = W.complex_gaussian(n, 960 + n)
    Z = A.copy()
    Z[n // 2, :] = 0
    assert gpu_c128(Z) == 0
    Z = A.copy()
    Z[:, n // 3] = 0
    _, _, asum = O.per(Z)
    T.check(gpu_c128(Z), 0.0, float(asum), n, T.unit(rows), f"zero column n={n}")
    R = W.real_gaussian(n, 961 + n)
    R[n - 1, :] = 0
    out = P.perm_f64(torch.from_numpy(R).cuda()).cpu().numpy()
    assert P.perm_last_status() == 0
    assert out[0] == 0


@pytest.mark.parametrize("n", [9, 17])
def test_unequal_entries_within_a_row(n, rows):
    """Entries spanning twelve orders of magnitude inside each row: the row
    scale follows the largest, the small entries keep their relative weight
    through the exact int64 (or double-float) columns."""
    A = W.complex_gaussian(n, 970 + n)
    mag = 10.0 ** np.random.default_rng(n).uniform(-6, 6, size=(n, n))
    B = A * mag
    re, im, asum = O.per(B)
    ref = complex(float(re), float(im))
    T.check(gpu_c128(B), ref, float(asum), n, T.unit(rows), f"unequal entries n={n}")


@pytest.mark.parametrize("n", [7, 9, 12])
def test_short_reseed_period_keeps_seed_precision(n, monkeypatch):
    """PERM_PDF_TILE_LOG=4: every row is re-seeded from its exact int64 value
    every 16 codes, so the conversion of the int64 seeds to double-float pairs
    (integer fields placed in FP32 significands, summed by FastTwoSum) sets the
    error.  It must stay at the double-float unit: |err| <= 8 n 2^-48 sum|t|.
    A dropped or misplaced 23-bit field of the conversion errs by about 2^-36
    per factor, which this bound rejects at these orders (few terms to average
    the error out).  Complex and real walks."""
    monkeypatch.setenv("PERM_PDF_TILE_LOG", "4")
    A = W.complex_gaussian(n, 990 + n)
    re, im, asum = O.per(A)
    err = abs(gpu_c128(A) - complex(float(re), float(im)))
    print(f"tile 16, complex n={n}: |err| / sum|t| = {err / float(asum):.3e}")
    assert err <= 8 * n * 2.0 ** -48 * float(asum)
    R = W.real_gaussian(n, 991 + n)
    re, _, asum = O.per(R)
    out = P.perm_f64(torch.from_numpy(R).cuda()).cpu().numpy()
    assert P.perm_last_status() == 0
    err = abs(float(out[0]) - float(re))
    print(f"tile 16, real n={n}: |err| / sum|t| = {err / float(asum):.3e}")
    assert err <= 8 * n * 2.0 ** -48 * float(asum)

"""Repeated columns on the GPU (perm_c128_repeated: the multiplicity classes of
Eq.(ryser2) summed in Glynn's halved form) against the oracle: its literal
evaluation of Eq.(ryser2), and its App. A walk over the expanded matrix
(the matrix with each column written out mult[k] times); plus closed forms.

Tolerances: against the oracle's walk of the expanded matrix, the 1e-10 bar
of tests/_tolerance.py (condition number from that walk's sum of term
magnitudes; merging equal terms leaves it unchanged).  The oracle's
Eq.(ryser2) is the un-halved sum, whose own rounding grows with the sum of
its term magnitudes, so that comparison allows max(1e-10 |per|,
8 n u sum|t|), u = 2^-53, sum|t| from the oracle.  One case at n = 30 (past
what the oracle finishes in seconds) is compared with the GPU walk of the
expanded matrix, at the bound its condition number allows."""
import math

import numpy as np
import pytest
import torch

import _tolerance as T
from oracle import oracle as O
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu
REL = 1e-10
U = 2.0 ** -53


def tol(n, ref, asum):
    return max(REL * abs(ref), 8 * n * U * float(asum))


def gpu_rep(Cb, mult):
    o = P.perm_c128_repeated(torch.from_numpy(np.ascontiguousarray(Cb.astype(np.complex128))).cuda(), mult)
    assert P.perm_last_status() == 0
    o = o.cpu().numpy()
    return complex(o[0], o[1])


@pytest.mark.parametrize("mult", [[1], [4], [1, 1], [2, 1, 3], [1] * 9, [3, 3, 3, 3], [5, 1, 1, 2, 6],
                                  [2] * 8, [7, 7, 6]])
def test_vs_oracle_ryser2(mult):
    n = sum(mult)
    Cb = W.haar_submatrix(n, n * n, 300 + n)[:, :len(mult)]
    r = O.per_repeated(Cb, mult)
    ref = complex(float(r[0]), float(r[1]))
    got = gpu_rep(Cb, mult)
    assert abs(got - ref) <= tol(n, ref, r[2]), (got, ref, float(r[2]))


def test_rows_of_extreme_magnitude():
    """Rows scaled by 1e+-300 and 2^+-1000: the products multiply unscaled row
    values and the rows' scales are applied once per thread, so no product
    chain leaves the double range; against the long-double oracle of the
    scaled matrix (its range reaches 1e+-4932)."""
    mult = [3, 1, 2, 2, 3]
    n = sum(mult)
    Cb = W.complex_gaussian(n, 331)[:, :len(mult)]
    s = np.ones(n)
    s[0], s[1], s[2], s[3] = 1e300, 1e-300, 2.0 ** 1000, 2.0 ** -1000
    Cb = Cb * s[:, None]
    r = O.per_repeated(Cb, mult)
    ref = complex(float(r[0]), float(r[1]))
    got = gpu_rep(Cb, mult)
    assert abs(got - ref) <= tol(n, ref, r[2]), (got, ref, float(r[2]))


@pytest.mark.parametrize("mult", [[3, 2, 2, 1, 4, 3, 2, 3, 2, 2], [1] * 18, [6, 6, 6, 4], [2] * 10])
def test_vs_oracle_walk_of_expanded(mult):
    n = sum(mult)
    Cb = (W.complex_gaussian(n, 7 + n) if len(mult) != 10 else W.haar_submatrix(n, n * n, 20))[:, :len(mult)]
    A = W.expand_columns(Cb, mult)
    re, im, asum = O.per(A)
    ref = complex(float(re), float(im))
    T.check(gpu_rep(Cb, mult), ref, float(asum), n, U, f"repeated columns {mult}")


def test_boson_sampling_collisions_n30():
    """15 modes with two photons each on a Haar S(900, 30) submatrix: the
    halved multiplicity form against the GPU Gray walk of the expanded matrix
    (the oracle needs minutes at n = 30; the same comparison against the
    oracle runs at n = 20 in test_vs_oracle_walk_of_expanded).  Merging equal
    terms leaves the condition number unchanged, about 4.6e5 for this input
    (sum of term magnitudes over |per|), beyond the reach of the 1e-10 bar:
    either result may be off by up to ~kappa n u = 1.5e-9; the bound allows
    1e-8."""
    Cb = W.haar_submatrix(30, 900, 30)[:, :15]
    A = W.expand_columns(Cb, [2] * 15)
    full = P.perm_c128(torch.from_numpy(A).cuda()).cpu().numpy()
    ref = complex(full[0], full[1])
    got = gpu_rep(Cb, [2] * 15)
    assert abs(got - ref) <= 1e-8 * abs(ref), (got, ref)


def test_closed_forms():
    for n in (1, 5, 12, 20):
        assert gpu_rep(np.ones((n, 1)), [n]) == pytest.approx(math.factorial(n), rel=1e-13)
    c = W.complex_gaussian(10, 4)[:, :1]
    ref = math.factorial(10) * np.prod(c[:, 0])
    assert abs(gpu_rep(c, [10]) - ref) <= 1e-13 * abs(ref)


def test_errors_and_host_buffers():
    Cb = W.complex_gaussian(6, 1)[:, :3]
    with pytest.raises(P.PermError):
        P.perm_c128_repeated(torch.from_numpy(Cb).cuda(), [2, 2, 1])  # sums to 5, not 6
    with pytest.raises(P.PermError):
        P.perm_c128_repeated(torch.from_numpy(Cb).cuda(), [2, 0, 4])
    host = P.perm_c128_repeated(torch.from_numpy(Cb), [2, 2, 2])
    torch.cuda.synchronize()
    assert host.device.type == "cpu"
    dev = P.perm_c128_repeated(torch.from_numpy(Cb).cuda(), [2, 2, 2]).cpu()
    assert torch.equal(host, dev)

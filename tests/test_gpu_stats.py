"""perm_batch_stats against the oracle: per-order counts, moments of
X = |per| / sqrt(n!) and the 16-bins-per-decade histogram, on a mixed batch
of circular (Sec. 4), Gaussian (Sec. 3) and Haar S(n^2.5, n) (Sec. 6)
matrices."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_stats_vs_oracle():
    rng = np.random.default_rng(17)
    mats, ns = [], []
    for k in range(1200):
        n = int(rng.integers(1, 15))
        kind = k % 3
        if kind == 0:
            A = W.circular(n, 40_000 + k)
        elif kind == 1:
            A = W.complex_gaussian(n, 40_000 + k)
        else:
            A = W.haar_submatrix(n, max(n, int(round(n ** 2.5))), 40_000 + k)
        mats.append(A)
        ns.append(n)
    dm = [torch.from_numpy(np.ascontiguousarray(A)).cuda() for A in mats]
    out, stats = P.perm_batch_stats(dm)
    assert P.perm_last_status() == 0
    st = stats.cpu().numpy()
    pers = []
    for A in mats:
        r = O.per(A)
        pers.append(complex(float(r[0]), float(r[1])))
    ref = O.batch_stats(pers, ns)
    assert np.array_equal(st[:, 0], ref[:, 0])
    for n in range(1, 15):
        for q in range(1, 5):
            assert st[n, q] == pytest.approx(ref[n, q], rel=1e-12), (n, q)
    # histograms: exact except for a value within rounding of a bin edge
    assert np.abs(st[:, 5:] - ref[:, 5:]).sum() <= 2
    assert st[:, 5:].sum() == len(mats)
    # second moment near 1 for the Gaussian-like families (loose)
    x2 = st[1:15, 2].sum() / st[1:15, 0].sum()
    assert 0.7 < x2 < 1.3


def test_stats_deterministic():
    mats = [torch.from_numpy(W.circular(10, s)).cuda() for s in range(300)]
    a = P.perm_batch_stats(mats)[1].cpu()
    b = P.perm_batch_stats(mats)[1].cpu()
    assert torch.equal(a, b)


def test_stats_many_chunks_of_one_order():
    """More results of one order than one block of the first statistics kernel
    takes (4096): 10,000 circular n = 5 matrices (three chunks) plus 5,000 of
    n = 3 (two chunks); the chunks' exact sums are added per order.  Counts and
    histograms against the oracle, moments at 1e-12."""
    mats, ns = [], []
    for k in range(10_000):
        mats.append(W.circular(5, 70_000 + k))
        ns.append(5)
    for k in range(5_000):
        mats.append(W.circular(3, 90_000 + k))
        ns.append(3)
    dm = [torch.from_numpy(np.ascontiguousarray(A)).cuda() for A in mats]
    out, stats = P.perm_batch_stats(dm)
    assert P.perm_last_status() == 0
    st = stats.cpu().numpy()
    o = out.cpu().numpy()
    # the oracle's statistics of the library's own permanents isolate the
    # statistics kernels (the permanents are checked elsewhere)
    ref = O.batch_stats([complex(a, b) for a, b in o], ns)
    assert np.array_equal(st[:, 0], ref[:, 0])
    for n in (3, 5):
        for q in range(1, 5):
            assert st[n, q] == pytest.approx(ref[n, q], rel=1e-12), (n, q)
    # histograms: exact except for a value within rounding of a bin edge
    assert np.abs(st[:, 5:] - ref[:, 5:]).sum() <= 2
    assert st[:, 5:].sum() == len(mats)

"""Batched permanents: each result against the single-matrix entry point and
the oracle; the statistics invariants of Sec. 3 as a loose systematic check."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(mats):
    dm = [torch.from_numpy(np.ascontiguousarray(m.astype(np.complex128))).cuda() for m in mats]
    out = P.perm_batch(dm)
    assert P.perm_last_status() == 0
    return out.cpu().numpy(), dm


def test_batch_vs_single_and_oracle(monkeypatch):
    """The batch walks exact fixed-point rows; each result equals a single
    perm_c128 launch with the same row arithmetic (PERM_ROWS=fixed) to
    rounding, and the oracle to 1e-10."""
    ns, mats = W.batch_study(300, seed=11, n_lo=1, n_hi=20)
    out, dm = _batch(mats)
    monkeypatch.setenv("PERM_ROWS", "fixed")
    for k in range(len(mats)):
        single = P.perm_c128(dm[k]).cpu().numpy()
        got = complex(out[k, 0], out[k, 1])
        one = complex(single[0], single[1])
        assert abs(got - one) <= 1e-12 * abs(one) + 1e-300
        if ns[k] <= 14 or k % 25 == 0:
            r = O.per(mats[k])
            ref = complex(float(r[0]), float(r[1]))
            assert abs(got - ref) <= 1e-10 * abs(ref)


def test_batch_config_shape_sample():
    """The batch study's distribution (n in 12..28, half Gaussian half Haar,
    shuffled) on a small sample, replayed twice through the cached graph."""
    ns, mats = W.batch_study(60, seed=3)
    out1, dm = _batch(mats)
    ptrs = torch.tensor([m.data_ptr() for m in dm], dtype=torch.int64).cuda()
    o = torch.empty((len(dm), 2), dtype=torch.float64, device="cuda")
    P.perm_batch(dm, out=o, ptrs=ptrs)
    P.perm_batch(dm, out=o, ptrs=ptrs)  # graph replay
    out2 = o.cpu().numpy()
    assert np.array_equal(out1, out2)
    for k in range(0, len(mats), 7):
        if ns[k] <= 24:
            r = O.per(mats[k])
            ref = complex(float(r[0]), float(r[1]))
            assert abs(complex(*out1[k]) - ref) <= 1e-10 * abs(ref)


def test_batch_moment_invariant():
    """Sec. 3: <|per|^2> = n! for variance-1 entries; 4000 Gaussian n=8 samples."""
    n, m = 8, 4000
    mats = [W.complex_gaussian(n, 10_000 + k) for k in range(m)]
    out, _ = _batch(mats)
    x2 = (out[:, 0] ** 2 + out[:, 1] ** 2) / math.factorial(n)
    # <X^2> = 1 and <X^4> = n + 1: the mean of X^2 within 5 standard errors
    se = math.sqrt((n + 1 - 1) / m)
    assert abs(x2.mean() - 1.0) < 5 * se


def test_batch_errors():
    with pytest.raises(P.PermError):
        P.perm_batch([torch.zeros((33, 33), dtype=torch.complex128, device="cuda")])

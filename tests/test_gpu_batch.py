"""Batched permanents: each result against the oracle (the 1e-10 bar of
tests/_tolerance.py) and against single launches of the same arithmetic;
each of the four batch kernels forced through the tuning table; a call on a
non-current stream; plan reuse with new pointers; the tuner; the statistics
invariants of Sec. 3 as a loose systematic check."""
import math

import numpy as np
import pytest
import torch

import _tolerance as T
from oracle import oracle as O
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_ORACLE = {}


def _oracle(A):
    key = np.asarray(A).tobytes()
    if key not in _ORACLE:
        r = O.per(A)
        _ORACLE[key] = (complex(float(r[0]), float(r[1])), float(r[2]))
    return _ORACLE[key]


def _dev(mats):
    return [torch.from_numpy(np.ascontiguousarray(m.astype(np.complex128))).cuda() for m in mats]


def _batch(mats, **kw):
    dm = _dev(mats)
    out = P.perm_batch(dm, **kw)
    assert P.perm_last_status() == 0
    return out.cpu().numpy(), dm


def _check_vs_oracle(out, ns, mats, every=1, n_max=20, what="batch"):
    for k in range(0, len(mats), every):
        if ns[k] <= n_max:
            ref, asum = _oracle(mats[k])
            T.check(complex(*out[k]), ref, asum, int(ns[k]), T.U_DF, f"{what} n={ns[k]} #{k}")


@pytest.fixture
def tuning():
    """Set the current device's tuning table for a test, restore it after."""
    saved = P.perm_batch_tuning(torch.cuda.current_device())

    def set_kinds(kind, L_warp=64, L_cta=64):
        L, K = [0] * 33, [0] * 33
        for n in range(1, 33):
            K[n] = kind
            L[n] = L_warp if kind == 1 else L_cta
        P.perm_batch_tuning(torch.cuda.current_device(), L, K)

    yield set_kinds
    P.perm_batch_tuning(torch.cuda.current_device(), *saved)


def test_batch_vs_oracle_and_single():
    """Default choices (warp kernel up to order 12, block kernels above): every
    result against the oracle, and against a single default launch."""
    ns, mats = W.batch_study(300, seed=11, n_lo=1, n_hi=20)
    out, dm = _batch(mats)
    _check_vs_oracle(out, ns, mats, every=1, n_max=14)
    _check_vs_oracle(out, ns, mats, every=7, n_max=20)
    for k in range(len(mats)):
        s = P.perm_c128(dm[k]).cpu().numpy()
        one = complex(s[0], s[1])
        assert abs(complex(*out[k]) - one) <= 1e-11 * abs(one) + 1e-300, (k, ns[k])


@pytest.mark.parametrize("kind", [1, 2, 3, 4])
def test_each_kernel_kind(kind, tuning):
    """All orders forced onto one kernel (1 warp per item, 2 block of 128
    threads per item, 3 the same at three blocks per SM, 4 block of 256
    threads per item), with chunks short enough that the larger matrices span
    several items."""
    tuning(kind, L_warp=16, L_cta=16)
    ns, mats = W.batch_study(120, seed=21 + kind, n_lo=1, n_hi=22)
    out, _ = _batch(mats)
    _check_vs_oracle(out, ns, mats, every=1, n_max=16, what=f"kind {kind}")
    _check_vs_oracle(out, ns, mats, every=5, n_max=22, what=f"kind {kind}")


def test_fixed_rows_match_single_fixed_launches(monkeypatch):
    """PERM_ROWS=fixed: every order on the warp kernel with exact fixed-point
    rows, equal to single launches of that arithmetic to rounding."""
    monkeypatch.setenv("PERM_ROWS", "fixed")
    ns, mats = W.batch_study(100, seed=12, n_lo=1, n_hi=20)
    out, dm = _batch(mats)
    for k in range(len(mats)):
        s = P.perm_c128(dm[k]).cpu().numpy()
        one = complex(s[0], s[1])
        assert abs(complex(*out[k]) - one) <= 1e-12 * abs(one) + 1e-300
    _check_vs_oracle(out, ns, mats, every=9)


@pytest.mark.parametrize("rows", ["pdf", "fixed"])
@pytest.mark.parametrize("kind", [0, 2])
def test_rows_of_extreme_magnitude(rows, kind, tuning, monkeypatch):
    """Rows scaled by 1e+-300 and 2^+-1000 on the built-in choices (warp kernel
    for the small orders) and forced onto the block kernel: each kernel applies
    the rows' scales once to an item's sum, so no product chain leaves the
    double range; against the long-double oracle of the scaled matrices."""
    monkeypatch.setenv("PERM_ROWS", rows)
    if kind:
        tuning(kind, L_cta=32)
    ns = [5, 8, 11, 14, 17]
    mats = []
    for k, n in enumerate(ns):
        A = W.complex_gaussian(n, 980 + k)
        s = np.ones(n)
        s[0], s[1], s[2], s[3] = 1e300, 1e-300, 2.0 ** 1000, 2.0 ** -1000
        mats.append(A * s[:, None])
    out, _ = _batch(mats)
    _check_vs_oracle(out, ns, mats, every=1, n_max=17, what=f"extreme rows {rows} kind {kind}")


def test_non_current_stream_without_pointer_tensor():
    """A batch launched on a stream other than the current one, with the
    pointer array and output made by the binding: results against the oracle
    after work on the current stream has reused freed memory."""
    ns, mats = W.batch_study(40, seed=13, n_lo=8, n_hi=18)
    dm = _dev(mats)
    s = torch.cuda.Stream()
    out = P.perm_batch(dm, stream=s)
    junk = [torch.full((1 << 16,), float(i), device="cuda") for i in range(8)]  # reuse of freed blocks
    s.synchronize()
    del junk
    o = out.cpu().numpy()
    _check_vs_oracle(o, ns, mats, every=1, n_max=18, what="side stream")


def test_plan_reused_with_new_pointers():
    """A second call with the same orders but other matrices and a new
    pointer tensor reuses the cached plan (no new plan is built) and returns
    the new matrices' permanents; a replay with the same pointers is bit
    identical."""
    ns, mats = W.batch_study(50, seed=14, n_lo=6, n_hi=18)
    out1, dm1 = _batch(mats)
    built = P.perm_batch_plans()
    mats2 = [W.complex_gaussian(int(n), 900 + k) for k, n in enumerate(ns)]
    out2, _ = _batch(mats2)
    assert P.perm_batch_plans() == built
    _check_vs_oracle(out2, ns, mats2, every=1, n_max=18, what="new pointers")
    out3 = P.perm_batch(dm1).cpu().numpy()
    assert np.array_equal(out1, out3)


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
    _check_vs_oracle(out1, ns, mats, every=7, n_max=24, what="study sample")


def test_autotune_fills_table(tuning):
    """perm_batch_autotune picks a kernel and a power-of-two chunk length for
    each order it times; batches then run on those choices correctly."""
    dev = torch.cuda.current_device()
    P.perm_batch_tuning(dev, [0] * 33, [0] * 33)
    P.perm_batch_autotune(10, 17)
    L, K = P.perm_batch_tuning(dev)
    print("tuned kinds", K[10:18], "lengths", L[10:18])
    for n in range(10, 18):
        assert K[n] in (1, 2, 3, 4) and L[n] >= 16 and (L[n] & (L[n] - 1)) == 0
    ns, mats = W.batch_study(60, seed=15, n_lo=10, n_hi=17)
    out, _ = _batch(mats)
    _check_vs_oracle(out, ns, mats, every=3, n_max=17, what="tuned")


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

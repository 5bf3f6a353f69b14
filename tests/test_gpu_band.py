"""App. C band permanents on the GPU (perm_c128_band) against the oracle's
exact-rational evaluation of the same recursion, the Gray-walk permanent,
and the Fibonacci closed form of the tridiagonal all-ones matrix."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1904_06229_gb300 import workloads as W
from paper_1904_06229_gb300 import perm as P

pytestmark = pytest.mark.gpu
REL = 1e-10


def gpu_band(A, k):
    o = P.perm_c128_band(torch.from_numpy(np.ascontiguousarray(A)).cuda(), k)
    assert P.perm_last_status() == 0
    o = o.cpu().numpy()
    return [complex(a, b) for a, b in o]


@pytest.mark.parametrize("n,k", [(1, 0), (1, 3), (3, 0), (6, 1), (9, 2), (12, 3), (14, 4), (16, 5), (30, 2),
                                 (40, 5)])
def test_vs_exact_oracle(n, k):
    A = W.band_matrix(n, k, 77 + n + k)
    br, bi = O.band_permanent_exact(A, k)
    ref = complex(float(br), float(bi))
    got = gpu_band(A, k)[0]
    assert abs(got - ref) <= REL * abs(ref), (got, ref)


@pytest.mark.parametrize("n,k", [(20, 3), (24, 5)])
def test_vs_gray_walk(n, k):
    A = W.band_matrix(n, k, n * k, kind="real")
    full = P.perm_c128(torch.from_numpy(A).cuda()).cpu().numpy()
    ref = complex(full[0], full[1])
    assert abs(gpu_band(A, k)[0] - ref) <= REL * abs(ref)


def test_fibonacci_and_batch():
    fib = [0, 1]
    for _ in range(100):
        fib.append(fib[-1] + fib[-2])
    mats = []
    for n in (2, 10, 50, 70):
        i, j = np.indices((n, n))
        mats.append(((np.abs(i - j) <= 1) * 1.0).astype(np.complex128))
        got = gpu_band(mats[-1], 1)[0]
        assert got == pytest.approx(fib[n + 1], rel=1e-14)
    # a batch of equal-size band matrices in one launch
    stack = np.stack([W.band_matrix(33, 4, s) for s in range(5)])
    out = gpu_band(stack, 4)
    for s in range(5):
        br, bi = O.band_permanent_exact(stack[s], 4)
        ref = complex(float(br), float(bi))
        assert abs(out[s] - ref) <= REL * abs(ref)


def test_long_band_matrix_runs():
    """n = 400, k = 5 (linear in n): zero the coupling between the two halves
    and compare with the product of the halves' permanents (block diagonal).
    Entries are scaled by 0.4 to keep |per| far from the double range limits."""
    n, h = 400, 200
    A = W.band_matrix(n, 5, 5) * 0.4
    A[h - 5:h, h:h + 5] = 0
    A[h:h + 5, h - 5:h] = 0
    whole = gpu_band(A, 5)[0]
    top = gpu_band(np.ascontiguousarray(A[:h, :h]), 5)[0]
    bot = gpu_band(np.ascontiguousarray(A[h:, h:]), 5)[0]
    assert np.isfinite(whole) and whole != 0
    assert abs(whole - top * bot) <= 1e-9 * abs(top * bot)


def test_errors():
    A = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(P.PermError):
        P.perm_c128_band(A, 6)
    with pytest.raises(P.PermError):
        P.perm_c128_band(A, -1)

"""App. B sparse permanents on the GPU (perm_c128_sparse) against the oracle
(its own greedy partition and sparsepermanent, and the dense Gray walk), on
the paper's sparse family: identity plus Bernoulli(p) off-diagonal entries.

Tolerance: the restricted sum is Ryser's un-halved form, so its FP64 accuracy
is bounded by the sum of its term magnitudes, max(1e-10 |per|, 8 n u sum|t|).
sum|t| is the same for every valid partition (a set J that misses every
non-zero of some row gives an exactly zero product), so the oracle's value,
computed with its own partition, bounds the library's sum as well."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1904_06229_gb300 import workloads as W
from paper_1904_06229_gb300 import perm as P

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def gpu_sparse(A):
    o = P.perm_c128_sparse(torch.from_numpy(np.ascontiguousarray(A)).cuda())
    assert P.perm_last_status() == 0
    o = o.cpu().numpy()
    return complex(o[0], o[1])


@pytest.mark.parametrize("n,p,seed", [(1, 0.5, 1), (4, 0.3, 2), (9, 0.2, 3), (13, 0.1, 4), (16, 0.1, 5),
                                      (18, 0.05, 6)])
def test_vs_oracle_sparse(n, p, seed):
    A = W.sparse_matrix(n, p, seed)
    r = O.per_sparse(A)  # the oracle's own partition: any valid partition gives per(A)
    ref = complex(float(r[0]), float(r[1]))
    got = gpu_sparse(A)
    assert abs(got - ref) <= max(1e-10 * abs(ref), 8 * n * U * float(r[2])), (got, ref, float(r[2]))


def test_rows_of_extreme_magnitude():
    """Rows scaled by 1e+-300 and 2^+-1000 (the products multiply unscaled row
    values, the rows' scales applied once per thread) against the long-double
    oracle of the scaled matrix."""
    n = 14
    A = W.sparse_matrix(n, 0.2, 41)
    s = np.ones(n)
    s[0], s[1], s[2], s[3] = 1e300, 1e-300, 2.0 ** 1000, 2.0 ** -1000
    A = A * s[:, None]
    r = O.per_sparse(A)
    ref = complex(float(r[0]), float(r[1]))
    got = gpu_sparse(A)
    assert abs(got - ref) <= max(1e-10 * abs(ref), 8 * n * U * float(r[2])), (got, ref, float(r[2]))


@pytest.mark.parametrize("n,p,seed", [(20, 0.1, 7), (24, 0.08, 8)])
def test_vs_glynn_oracle(n, p, seed):
    A = W.sparse_matrix(n, p, seed)
    g = O.per(A)
    ref = complex(float(g[0]), float(g[1]))
    assert abs(gpu_sparse(A) - ref) <= 1e-9 * abs(ref)


def test_vs_dense_walk_n32():
    A = W.sparse_matrix(32, 0.04, 32)
    d = P.perm_c128(torch.from_numpy(A).cuda()).cpu().numpy()
    ref = complex(d[0], d[1])
    assert abs(gpu_sparse(A) - ref) <= 1e-9 * abs(ref)


def test_identity_permutation_and_blocks():
    assert gpu_sparse(np.eye(20, dtype=complex)) == 1
    Pm = np.eye(30, dtype=complex)[np.random.default_rng(4).permutation(30)]
    assert gpu_sparse(Pm) == 1
    B = W.sparse_matrix(10, 0.2, 1)
    C = W.sparse_matrix(9, 0.2, 2)
    M = np.zeros((19, 19), dtype=complex)
    M[:10, :10] = B
    M[10:, 10:] = C
    pb, pc = O.per(B), O.per(C)
    ref = complex(float(pb[0]), float(pb[1])) * complex(float(pc[0]), float(pc[1]))
    asum = float(O.per_sparse(M)[2])
    assert abs(gpu_sparse(M) - ref) <= max(1e-10 * abs(ref), 8 * 19 * U * asum)


def test_large_sparse_runs():
    """n = 48, p = 0.02: 2^25 sets instead of 2^47."""
    A = W.sparse_matrix(48, 0.02, 48)
    block, count = P.perm_sparse_partition(A)
    assert 0 < count < 1 << 30
    v = gpu_sparse(A)
    assert np.isfinite(v.real) and np.isfinite(v.imag) and v != 0

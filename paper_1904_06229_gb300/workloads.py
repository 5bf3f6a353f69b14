"""Seeded synthetic inputs shaped like the paper's random-matrix workloads.

This module is shared by the tests, the benchmark and the oracle-side checks.
It holds input generation only: none of the permanent's arithmetic.

Generators (paper sections they follow):
  complex_gaussian  Sec. 3: entries (g1 + i g2)/sqrt(2), g1, g2 ~ N(0,1)
                    (the Ginibre ensemble G(n)); the real block is drawn first.
  haar_submatrix    Sec. 6: S = sqrt(m) * (top-left n x n block of a Haar unitary
                    of order m), the unitary from a QR factorisation of a complex
                    Gaussian matrix with the phase fix lambda_ii = r_ii/|r_ii|.
                    Only the first n columns of U enter the top-left block, and
                    they depend only on the first n columns of the Gaussian
                    matrix, so a thin QR of an m x n Gaussian block gives the
                    same distribution at O(m n^2) cost.
  circular          Sec. 4: entries exp(i theta), theta ~ U[0, 2 pi).
  real_gaussian     real N(0,1) entries.
  bernoulli_pm1     Sec. 5: entries +-1 with probability 1/2.
  zero_one          0-1 entries with a given density.
  batch_study       the many-matrix study: n ~ U{n_lo..n_hi}, alternating
                    Gaussian / Haar (m = n^2) members, shuffled order.
  sparse_matrix     Sec. 2.D / App. B timing family: identity plus
                    Bernoulli(p) off-diagonal non-zeros (complex Gaussian values).
  band_matrix       Sec. 2.D / App. C: zero outside |i - j| <= k.
  expand_columns    the n x n matrix with column k of a given n x R matrix
                    repeated mult[k] times (Eq. ryser2 inputs).
All draws use numpy's PCG64 (`numpy.random.default_rng(seed)`).
"""
from __future__ import annotations

import numpy as np


def complex_gaussian(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n, n))
    im = rng.standard_normal((n, n))
    return (re + 1j * im) * np.sqrt(0.5)


def haar_submatrix(n: int, m: int | None = None, seed: int | None = None) -> np.ndarray:
    if m is None:
        m = n * n
    if seed is None:
        seed = 1000 + n
    if m < n:
        raise ValueError("m >= n required")
    rng = np.random.default_rng(seed)
    g = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) * np.sqrt(0.5)
    q, r = np.linalg.qr(g, mode="reduced")
    d = np.diag(r)
    lam = d / np.abs(d)
    u = q * lam[None, :]
    return np.sqrt(m) * u[:n, :n]


def circular(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 2.0 * np.pi, (n, n))
    return np.exp(1j * th)


def real_gaussian(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal((n, n))


def bernoulli_pm1(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.where(rng.random((n, n)) < 0.5, -1, 1).astype(np.int8)


def zero_one(n: int, seed: int, density: float = 0.5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.random((n, n)) < density).astype(np.int8)


def batch_sizes(count: int, seed: int, n_lo: int = 12, n_hi: int = 28) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(n_lo, n_hi + 1, size=count)


def batch_study(count: int, seed: int = 3, n_lo: int = 12, n_hi: int = 28):
    """Return (ns, mats): ns[k] the order of matrix k, mats[k] a complex128
    n x n array.  Even positions of the unshuffled list are Gaussian G(n),
    odd ones Haar S(n^2, n); the list is then shuffled with the same seed."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    mats = []
    for k, n in enumerate(ns):
        n = int(n)
        sub = int(rng.integers(0, 2**62))
        if k % 2 == 0:
            mats.append(complex_gaussian(n, sub))
        else:
            mats.append(haar_submatrix(n, n * n, sub))
    order = rng.permutation(count)
    return ns[order], [mats[i] for i in order]


def sparse_matrix(n: int, p: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < p
    np.fill_diagonal(mask, True)
    vals = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * np.sqrt(0.5)
    return np.where(mask, vals, 0).astype(np.complex128)


def band_matrix(n: int, k: int, seed: int, kind: str = "gaussian") -> np.ndarray:
    """Random band matrix; kind='real' gives real N(0,1) entries (the App. C
    timing study), otherwise complex Gaussian."""
    rng = np.random.default_rng(seed)
    if kind == "real":
        A = rng.standard_normal((n, n)).astype(np.complex128)
    else:
        A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * np.sqrt(0.5)
    i, j = np.indices((n, n))
    A[np.abs(i - j) > k] = 0
    return A


def expand_columns(Cbar, mult) -> np.ndarray:
    Cb = np.asarray(Cbar)
    return np.concatenate([np.repeat(Cb[:, k:k + 1], int(mk), axis=1) for k, mk in enumerate(mult)], axis=1)

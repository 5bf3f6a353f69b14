"""FP32-product variant: error against the FP64 oracle within the bound the
arithmetic gives (each factor rounded to 24 bits, n-1 FP32 multiplies:
relative error per term <= (2n + 2) 2^-24; summed over terms:
|err| <= (2n + 2) 2^-24 * Sigma|t|), and the observed error is reported."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(autouse=True, params=["fixed", "fp64"])
def rows(request, monkeypatch):
    monkeypatch.setenv("PERM_ROWS", request.param)
    return request.param


def _bound(n, asum):
    return (2 * n + 2) * U32 * asum


@pytest.mark.parametrize("n", [1, 2, 3, 6, 11, 16, 21])
def test_c128_f32p_within_bound(n):
    A = W.complex_gaussian(n, 800 + n)
    r = O.per(A)
    ref = complex(float(r[0]), float(r[1]))
    o = P.perm_c128_f32p(torch.from_numpy(A).cuda()).cpu().numpy()
    got = complex(o[0], o[1])
    assert abs(got - ref) <= _bound(n, float(r[2]))


@pytest.mark.parametrize("n", [1, 4, 12, 20, 24])
def test_f64_f32p_within_bound(n):
    A = W.real_gaussian(n, 900 + n)
    r = O.per(A)
    got = float(P.perm_f64_f32p(torch.from_numpy(A).cuda()).cpu().numpy()[0])
    assert abs(got - float(r[0])) <= _bound(n, float(r[2]))


def test_config_real_gaussian_n32_vs_fp64():
    """Precision study: real N(0,1) n = 32 (seed 4), FP32 products against the
    FP64 path (both are checked against the stored oracle value in
    test_gpu_golden.py); the relative difference is reported."""
    A = W.real_gaussian(32, 4)
    t = torch.from_numpy(A).cuda()
    f64 = float(P.perm_f64(t).cpu().numpy()[0])
    f32p = float(P.perm_f64_f32p(t).cpu().numpy()[0])
    rel = abs(f32p - f64) / abs(f64)
    print(f"n=32 real Gaussian: FP64 {f64!r} FP32-product {f32p!r} rel diff {rel:.3e}")
    assert rel < 1e-4


def test_config_pm1_n30_exact_reference():
    """Precision study: +-1 n = 30 (seed 5) against the exact integer."""
    A = W.bernoulli_pm1(30, 5)
    ex = O.per_exact(A, parts=4096)
    t = torch.from_numpy(A.astype(np.float64)).cuda()
    f64 = float(P.perm_f64(t).cpu().numpy()[0])
    f32p = float(P.perm_f64_f32p(t).cpu().numpy()[0])
    e64 = abs(f64 - ex) / abs(ex)
    e32 = abs(f32p - ex) / abs(ex)
    print(f"+-1 n=30: exact {ex} FP64 rel {e64:.3e} FP32-product rel {e32:.3e}")
    assert e64 < 1e-10

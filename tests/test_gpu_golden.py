"""Full-size seeded configurations against stored oracle values
(tests/golden/configs.json, written by tests/golden/make_golden.py from the
oracle alone):

  * exact 0-1 permanents, density 1/2, n = 30 (seed 6) and n = 36 (seed 7),
    and the +-1 n = 30 (seed 5) precision-study matrix: perm_mod01 modulo the
    four 62-bit primes plus perm_crt, bit for bit against the oracle's
    512-bit integer walk, in both of the library's summation modes (exact
    per-thread sums, and the modular group walk);
  * real N(0,1) n = 32 (seed 4): perm_f64 at the 1e-10 bar and the FP32-
    product variant perm_f64_f32p within its stated bound
    (2n + 2) 2^-24 sum|t|, sum|t| from the oracle;
  * +-1 n = 30: perm_f64 against the exact integer at 1e-10, and the FP32-
    product variant within its stated bound.

The stored matrices themselves are used (the CPU test test_golden_cpu.py
checks that the generators still produce them).
"""
import json
import os

import numpy as np
import pytest
import torch

import _tolerance as T
from paper_1904_06229_gb300 import perm as P

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
U32 = 2.0 ** -24


def cases():
    with open(os.path.join(HERE, "golden", "configs.json")) as f:
        return json.load(f)["cases"]


def matrix(case):
    if case["kind"] == "exact":
        return np.array([[int(v) for v in row.split()] for row in case["matrix"]], dtype=np.int8)
    return np.array([[float.fromhex(v) for v in row.split()] for row in case["matrix"]], dtype=np.float64)


@pytest.mark.parametrize("summation", ["exact", "modular"])
@pytest.mark.parametrize("name", ["zero_one_n30_seed6", "zero_one_n36_seed7", "pm1_n30_seed5"])
def test_exact_config_bit_exact(name, summation, monkeypatch):
    if summation == "modular":
        monkeypatch.setenv("PERM_MOD_SUM", "modular")
    case = cases()[name]
    A = torch.from_numpy(matrix(case)).cuda()
    primes = P.perm_default_primes()
    res = P.perm_mod01(A, primes)
    assert P.perm_last_status() == 0
    got = P.perm_crt([int(v) for v in res.cpu()], primes)
    print(f"{name} ({summation} sums): GPU {got} oracle {case['per']}")
    assert got == int(case["per"])


def test_real_gaussian_n32_fp64_and_f32p():
    case = cases()["real_gaussian_n32_seed4"]
    A = torch.from_numpy(matrix(case)).cuda()
    ref = float(case["per"])
    asum = float(case["abs_sum"])
    f64 = float(P.perm_f64(A).cpu().numpy()[0])
    T.check(f64, ref, asum, 32, T.U64, "real Gaussian n=32, perm_f64")
    f32p = float(P.perm_f64_f32p(A).cpu().numpy()[0])
    bound = (2 * 32 + 2) * U32 * asum
    print(f"real Gaussian n=32, perm_f64_f32p: rel err {abs(f32p - ref) / abs(ref):.3e}, "
          f"stated bound {bound / abs(ref):.3e} relative")
    assert abs(f32p - ref) <= bound


def test_pm1_n30_fp64_and_f32p():
    case = cases()["pm1_n30_seed5"]
    A = torch.from_numpy(matrix(case).astype(np.float64)).cuda()
    ex = int(case["per"])
    asum = float(case["abs_sum"])
    f64 = float(P.perm_f64(A).cpu().numpy()[0])
    T.check(f64, float(ex), asum, 30, T.U64, "+-1 n=30, perm_f64")
    f32p = float(P.perm_f64_f32p(A).cpu().numpy()[0])
    bound = (2 * 30 + 2) * U32 * asum
    print(f"+-1 n=30, perm_f64_f32p: rel err {abs(f32p - ex) / abs(ex):.3e}, "
          f"stated bound {bound / abs(ex):.3e} relative")
    assert abs(f32p - ex) <= bound

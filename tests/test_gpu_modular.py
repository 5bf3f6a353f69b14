"""GPU exact path (perm_mod01 + host CRT) against the oracle's exact integer
and modular forms: bit-exact residues and integers."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRIMES = O.default_primes()

# The kernel sums exactly in 192- or 256-bit integers where the bound allows
# it and otherwise multiplies row groups modulo each prime; PERM_MOD_SUM=modular
# forces the second form so both are checked at the same sizes.
SUMS = ["auto", "modular"]


@pytest.fixture(params=SUMS)
def mod_sum(request, monkeypatch):
    if request.param == "modular":
        monkeypatch.setenv("PERM_MOD_SUM", "modular")
    else:
        monkeypatch.delenv("PERM_MOD_SUM", raising=False)
    return request.param


def gpu_mod(A, primes=PRIMES):
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.int8))).cuda()
    r = P.perm_mod01(t, primes).cpu().numpy()
    return [int(v) for v in r]


def gpu_exact(A):
    return P.perm_crt(gpu_mod(A), PRIMES)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 9, 12, 16, 17, 20])
def test_zero_one_and_pm1_exact(n, mod_sum):
    for A in (W.zero_one(n, 600 + n), W.bernoulli_pm1(n, 650 + n)):
        ex = O.per_exact(A)
        assert gpu_mod(A) == [ex % p for p in PRIMES]
        assert gpu_exact(A) == ex


@pytest.mark.parametrize("n", [5, 9, 13])
def test_general_int8_exact(n, mod_sum):
    """Entries up to +-127 take the 4-row grouping of the exact products."""
    A = np.random.default_rng(n).integers(-127, 128, (n, n)).astype(np.int8)
    ex = O.per_exact(A)
    assert gpu_exact(A) == ex
    assert gpu_mod(A) == O.per_mod(A, PRIMES)


def test_closed_forms(mod_sum):
    for n in (10, 20, 25):
        J = np.ones((n, n), dtype=np.int8)
        import math

        assert gpu_exact(J) == math.factorial(n)
        D = [1, 0]
        for k in range(2, n + 1):
            D.append((k - 1) * (D[-1] + D[-2]))
        assert gpu_exact(J - np.eye(n, dtype=np.int8)) == D[n]
        assert gpu_exact(np.eye(n, dtype=np.int8)) == 1


def test_other_moduli():
    A = W.zero_one(14, 3)
    ps = O.largest_primes_below(1 << 40, 4)
    assert gpu_mod(A, ps) == O.per_mod(A, ps)


@pytest.mark.parametrize(
    "moduli",
    [
        [3, 5, 7, 11],  # every group product exceeds the moduli
        [1000003, 999983, 65537, 257],
        "below 2^40",
        "below 2^52",
    ],
)
@pytest.mark.parametrize("kind", ["zero_one", "pm1", "int8", "small"])
def test_moduli_smaller_than_group_products(moduli, kind, mod_sum):
    """Any odd moduli below 2^62 are accepted; where a row group's product can
    exceed the smallest modulus the kernel reduces groups through R^2.  The
    residues are compared with the exact permanent reduced in Python."""
    if moduli == "below 2^40":
        moduli = O.largest_primes_below(1 << 40, 4)
    elif moduli == "below 2^52":
        moduli = O.largest_primes_below(1 << 52, 4)
    n = 13
    rng = np.random.default_rng(len(kind) * 7 + n)
    A = {
        "zero_one": W.zero_one(n, 91),
        "pm1": W.bernoulli_pm1(n, 92),
        # n = 24 with entries up to 127: sums need more than 256 bits, so
        # this one takes the modular group walk even without the override
        "int8": np.random.default_rng(24).integers(-127, 128, (24, 24)).astype(np.int8),
        "small": rng.integers(0, 4, (n, n)).astype(np.int8),
    }[kind]
    ex = O.per_exact(A)
    assert gpu_mod(A, moduli) == [ex % p for p in moduli]


@pytest.mark.parametrize("n", [1, 2, 11, 12, 13, 24, 25])
def test_group_size_boundaries(n, mod_sum):
    """Orders on both sides of the 12-, 8- and 4-row groups; entries 0..3 make
    rows sums up to 3n, so the 8-row grouping is taken where 12 rows would
    overflow the moduli."""
    A = np.random.default_rng(500 + n).integers(0, 4, (n, n)).astype(np.int8)
    ex = O.per_exact(A)
    assert gpu_mod(A) == [ex % p for p in PRIMES]
    assert gpu_exact(A) == ex


def test_exact_sum_widths():
    """Cases for each exact-sum form: 256-bit sums with 6-row int32 factors
    (all-ones and J - I at n = 35: n! and the derangement number), 256-bit sums
    with 2-row factors (entries up to 127, n = 20), 192-bit with 2-row factors
    (n = 12)."""
    import math

    J = np.ones((35, 35), dtype=np.int8)
    assert gpu_exact(J) == math.factorial(35)
    D = [1, 0]
    for k in range(2, 36):
        D.append((k - 1) * (D[-1] + D[-2]))
    assert gpu_exact(J - np.eye(35, dtype=np.int8)) == D[35]
    for n in (12, 20):
        A = np.random.default_rng(700 + n).integers(-127, 128, (n, n)).astype(np.int8)
        ex = O.per_exact(A)
        assert gpu_mod(A) == [ex % p for p in PRIMES]
        assert gpu_exact(A) == ex


def test_both_sums_agree_n28(monkeypatch):
    """0-1 n = 28: the exact-integer sum and the modular group walk give the
    same residues."""
    A = W.zero_one(28, 13)
    monkeypatch.delenv("PERM_MOD_SUM", raising=False)
    a = gpu_mod(A)
    monkeypatch.setenv("PERM_MOD_SUM", "modular")
    b = gpu_mod(A)
    assert a == b


def test_config_n30_zero_one():
    """0-1 density 1/2, n = 30, seed 6: bit-exact against the 512-bit oracle."""
    A = W.zero_one(30, 6)
    ex = O.per_exact(A, parts=4096)
    got = gpu_exact(A)
    print(f"n=30 0-1 seed6 per = {got}")
    assert got == ex


def test_config_n36_block_diagonal():
    """n = 36 at full size: per(diag(B, C)) = per(B) per(C) exactly."""
    B = W.zero_one(18, 71)
    C = W.zero_one(18, 72)
    M = np.zeros((36, 36), dtype=np.int8)
    M[:18, :18] = B
    M[18:, 18:] = C
    ref = O.per_exact(B) * O.per_exact(C)
    assert gpu_exact(M) == ref
    # and under a row/column permutation
    rng = np.random.default_rng(1)
    assert gpu_exact(M[rng.permutation(36)][:, rng.permutation(36)]) == ref


def test_pm1_n30_config():
    """+-1 Bernoulli n = 30, seed 5 (the precision study's exact reference)."""
    A = W.bernoulli_pm1(30, 5)
    ex = O.per_exact(A, parts=4096)
    assert gpu_exact(A) == ex


def test_host_buffers():
    A = W.zero_one(11, 1)
    t = torch.from_numpy(A)
    out = torch.empty(4, dtype=torch.int64)
    P.perm_mod01(t, PRIMES, out)
    torch.cuda.synchronize()
    assert [int(v) for v in out] == gpu_mod(A)

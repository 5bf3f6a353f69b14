"""The stored full-size oracle values (tests/golden/configs.json, written by
tests/golden/make_golden.py from the oracle alone): every configuration is
present, the seeded generators still produce the stored matrices, and the
stored values are consistent with what the paper and the mathematics fix
(exact values are integers of the right parity class, the real value's
magnitude is below its sum of term magnitudes)."""
import json
import os

import numpy as np

from paper_1904_06229_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "configs.json")

GENERATORS = {
    "zero_one_n36_seed7": lambda: W.zero_one(36, 7),
    "zero_one_n30_seed6": lambda: W.zero_one(30, 6),
    "pm1_n30_seed5": lambda: W.bernoulli_pm1(30, 5),
    "real_gaussian_n32_seed4": lambda: W.real_gaussian(32, 4),
}


def load_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def stored_matrix(case):
    if case["kind"] == "exact":
        return np.array([[int(v) for v in row.split()] for row in case["matrix"]], dtype=np.int8)
    return np.array([[float.fromhex(v) for v in row.split()] for row in case["matrix"]], dtype=np.float64)


def test_every_configuration_is_stored():
    cases = load_cases()
    assert set(GENERATORS) <= set(cases)


def test_generators_reproduce_stored_matrices():
    cases = load_cases()
    for name, gen in GENERATORS.items():
        A = gen()
        B = stored_matrix(cases[name])
        assert A.shape == B.shape == (cases[name]["n"], cases[name]["n"])
        assert np.array_equal(A.astype(B.dtype), B), name


def test_stored_values_consistent():
    cases = load_cases()
    for name in ("zero_one_n36_seed7", "zero_one_n30_seed6"):
        v = int(cases[name]["per"])
        # a 0-1 permanent counts perfect matchings: a non-negative integer,
        # at most the product of the row sums (Minc-Bregman's weaker form)
        A = stored_matrix(cases[name]).astype(np.int64)
        assert 0 <= v <= int(np.prod([int(s) for s in A.sum(axis=1)], dtype=object))
        assert v.bit_length() == cases[name]["per_bits"]
    v = int(cases["pm1_n30_seed5"]["per"])
    # every term of a +-1 permanent is +-1: per = n! (mod 2), n! even
    assert v % 2 == 0 and abs(v) <= __import__("math").factorial(30)
    c = cases["real_gaussian_n32_seed4"]
    assert abs(float(c["per"])) <= float(c["abs_sum"])
    assert float(c["per_im"]) == 0.0

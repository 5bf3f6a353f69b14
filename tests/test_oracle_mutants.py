"""Mutation test of the oracle's pins: six plausible mistakes are planted in
the oracle's Gray-code walk (a dropped term, a sign never flipped, a wrong
column index, a transposed operand, a missing halving, the wrong final sign),
each compiled as its own library on the CPU; every mutant must fail at least
one pin that the correct oracle passes."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_06229_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "perm_oracle.c")


def _build(k, tmp):
    out = os.path.join(tmp, f"liboracle_mut{k}.so")
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", f"-DORACLE_MUTANT={k}",
                    "-o", out, SRC], check=True)
    lib = ctypes.CDLL(out)
    lib.oracle_per_glynn_c.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p]
    return lib


def _per(lib, A):
    a = np.ascontiguousarray(np.asarray(A, dtype=np.complex128)).view(np.float64)
    out = np.zeros(2, dtype=np.longdouble)
    s = np.zeros(1, dtype=np.longdouble)
    assert lib.oracle_per_glynn_c(a.ctypes.data, a.shape[0], 4, 1, out.ctypes.data, s.ctypes.data) == 0
    return complex(float(out[0]), float(out[1]))


def _pins():
    """(matrix, exact value) pairs the correct oracle reproduces."""
    cases = []
    for n in (3, 5):
        A = W.complex_gaussian(n, 900 + n)
        er, ei = O.per_brute_exact(A)
        cases.append((A, complex(float(er), float(ei))))
    cases.append((np.ones((4, 4)), 24.0))                       # per(J_4) = 4!
    cases.append((np.ones((5, 5)) - np.eye(5), 44.0))           # derangements D_5
    cases.append((np.array([[1, 2, 3], [4, 5, 6], [7, 8, 9]], dtype=float), 450.0))
    return cases


def _fails(lib):
    for A, ref in _pins():
        got = _per(lib, A)
        if not abs(got - ref) <= 1e-12 * max(1.0, abs(ref)):
            return True
    return False


def test_correct_oracle_passes_the_pins(tmp_path):
    assert not _fails(_build(0, str(tmp_path)))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_every_planted_mistake_is_caught(k, tmp_path):
    assert _fails(_build(k, str(tmp_path))), f"mutant {k} passed every pin"

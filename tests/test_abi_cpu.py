"""C ABI checks that need no GPU: the library builds and loads, exports every
symbol include/perm.h declares, and its host-only helpers (prime search,
Chinese remaindering, status strings) behave; compute calls without a device
fail with PERM_ECUDA instead of falling back to the CPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1904_06229_gb300 import build, perm

    build.build()
    return perm.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "perm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(perm_\w+)\s*\(", txt, re.M)))


def test_header_matches_binding_list():
    from paper_1904_06229_gb300 import perm

    assert _declared() == sorted(perm.EXPORTS)


def test_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_no_cuda_runtime_dependency(lib):
    from paper_1904_06229_gb300 import perm

    # the runtime is linked statically; only the driver is needed at run time
    maps = open("/proc/self/maps").read()
    assert perm.LIB_PATH in maps


def test_default_primes_match_oracle(lib):
    from oracle import oracle as O
    from paper_1904_06229_gb300 import perm

    assert perm.perm_default_primes() == O.default_primes()


def test_crt_host(lib):
    from oracle import oracle as O
    from paper_1904_06229_gb300 import perm

    ps = perm.perm_default_primes()
    for v in (0, 1, -1, 12345678901234567890, -(3**150), (1 << 240) - 7):
        assert perm.perm_crt([v % p for p in ps], ps) == v
        assert perm.perm_crt([v % p for p in ps], ps) == O.crt([v % p for p in ps], ps)
    # fewer moduli
    assert perm.perm_crt([5 % ps[0]], ps[:1]) == 5
    assert perm.perm_crt([(-5) % ps[0], (-5) % ps[1]], ps[:2]) == -5


def test_crt_errors(lib):
    from paper_1904_06229_gb300 import perm

    with pytest.raises(perm.PermError) as e:
        perm.perm_crt([1, 2], [7, 7])
    assert e.value.code == -7
    with pytest.raises(perm.PermError) as e:
        perm.perm_crt([9], [7])
    assert e.value.code == -1


def test_status_strings(lib):
    from paper_1904_06229_gb300 import perm

    for code, name in perm.STATUS.items():
        assert perm.perm_status_string(code).startswith(name)


def test_argument_errors_before_device(lib):
    """Argument errors are reported before any CUDA call."""
    vp = ctypes.c_void_p
    buf = (ctypes.c_double * 8)()
    a = ctypes.addressof(buf)
    assert lib.perm_c128(None, 3, a, None) == -2
    assert lib.perm_c128(a, 0, a, None) == -1
    assert lib.perm_c128(a, 65, a, None) == -1
    assert lib.perm_f64(a, -1, a, None) == -1
    assert lib.perm_c128_range(a, 3, 4, 1, a, None) == -1  # past 2^(n-1)
    assert lib.perm_c128_range(a, 3, 0, 5, a, None) == -1
    pr = (ctypes.c_uint64 * 4)(7, 11, 13, 13)
    assert lib.perm_mod01(a, 3, ctypes.addressof(pr), a, None) == -7
    pr = (ctypes.c_uint64 * 4)(7, 11, 13, 1 << 62)
    assert lib.perm_mod01(a, 3, ctypes.addressof(pr), a, None) == -7
    pr = (ctypes.c_uint64 * 4)(7, 11, 13, 16)
    assert lib.perm_mod01(a, 3, ctypes.addressof(pr), a, None) == -7
    # band: sizes whose byte count would not be addressable
    assert lib.perm_c128_band(a, 65535, 2, 1 << 30, a, None) == -1
    assert lib.perm_c128_band(a, 65535, 2, 4097, a, None) == -1
    assert lib.perm_c128_band(a, 10, 6, 1, a, None) == -1
    assert lib.perm_c128_band(a, 10, 2, 0, a, None) == -1


def test_no_cpu_fallback_without_device(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("device present")
    buf = (ctypes.c_double * 8)(1, 0, 0, 0, 0, 0, 0, 0)
    out = (ctypes.c_double * 2)()
    assert lib.perm_c128(ctypes.addressof(buf), 1, ctypes.addressof(out), None) == -3
    assert lib.perm_f64(ctypes.addressof(buf), 1, ctypes.addressof(out), None) == -3
    assert lib.perm_last_status(None) == -3
    v = ctypes.c_double()
    assert lib.perm_fp64_peak(ctypes.addressof(v)) == -3


def test_sparse_partition_host(lib):
    """The library's greedy partition (host-only): pairwise-disjoint row
    neighbourhoods, the App. B set count, never worse than the first-choice
    greedy pass of the oracle's independent implementation."""
    import math

    import numpy as np

    from oracle import oracle as O
    from paper_1904_06229_gb300 import perm
    from paper_1904_06229_gb300 import workloads as W

    for n, p, seed in ((30, 0.05, 1), (48, 0.02, 2), (64, 0.005, 3), (5, 0.9, 4)):
        A = W.sparse_matrix(n, p, seed)
        block, count = perm.perm_sparse_partition(A)
        nb = max(block) + 1
        rows = [set(np.nonzero(A[i])[0].tolist()) for i in range(n)]
        for l in range(nb):
            S = {j for j in range(n) if block[j] == l}
            assert S and S in rows
        assert count == O.partition_count(block)
        assert count <= O.partition_count(O.greedy_partition(A))
        assert math.log2(count) <= n


def test_fault_injection_plan_stage(lib, monkeypatch):
    """PERM_FAULT=plan makes a walk call fail as if its scratch could not be
    had (PERM_ENOMEM), before any device work; "plan:k" fails only the k-th
    call that reaches that step."""
    buf = (ctypes.c_double * 8)(1, 0, 0, 0, 0, 0, 0, 0)
    out = (ctypes.c_double * 4)()
    a, o = ctypes.addressof(buf), ctypes.addressof(out)
    monkeypatch.setenv("PERM_FAULT", "plan")
    assert lib.perm_c128(a, 1, o, None) == -6
    assert lib.perm_f64_range(a, 1, 0, 1, o, None) == -6
    monkeypatch.setenv("PERM_FAULT", "plan:2")
    codes = [lib.perm_c128(a, 1, o, None) for _ in range(3)]
    assert codes[1] == -6 and codes[0] != -6 and codes[2] != -6
    monkeypatch.setenv("PERM_FAULT", "launch")  # other stages leave this step alone
    assert lib.perm_c128(a, 1, o, None) != -6
    monkeypatch.delenv("PERM_FAULT")
    assert lib.perm_c128(a, 1, o, None) != -6

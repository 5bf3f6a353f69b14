"""perm_c128_noalloc, the variant for callers that cannot allocate device
memory (it keeps its partial sums in a static array inside the library),
called through the C ABI on two calls in a row and compared with perm_c128
and with the CPU oracle.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import _tolerance as T
from oracle import oracle as O
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = T.REL  # the FP64 parity tolerance of the other tests


def _call(lib, A, n, out):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.perm_c128_noalloc(ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream))


@pytest.mark.parametrize("n,seed", [(1, 3), (12, 4), (20, 0), (27, 5)])
def test_noalloc_matches_perm_c128_twice(n, seed):
    lib = P.load()
    A = torch.from_numpy(W.complex_gaussian(n, seed)).cuda()
    ref = P.perm_c128(A).cpu().numpy()
    refc = complex(ref[0], ref[1])
    re, im, asum = O.per(W.complex_gaussian(n, seed))
    oracle = complex(float(re), float(im))
    for _ in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, A, n, out) == 0
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        got = complex(o[0], o[1])
        assert abs(got - refc) <= REL * abs(refc), (n, got, refc)
        T.check(got, oracle, float(asum), n, T.U_DF, f"perm_c128_noalloc n={n}")


def test_noalloc_rejects_bad_arguments():
    lib = P.load()
    A = torch.from_numpy(W.complex_gaussian(4, 1)).cuda()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    assert _call(lib, A, 0, out) == -1
    assert _call(lib, A, 65, out) == -1
    host = torch.from_numpy(W.complex_gaussian(4, 1))
    assert lib.perm_c128_noalloc(ctypes.c_void_p(host.data_ptr()), 4, ctypes.c_void_p(out.data_ptr()), None) == -1
    assert lib.perm_c128_noalloc(None, 4, ctypes.c_void_p(out.data_ptr()), None) == -2

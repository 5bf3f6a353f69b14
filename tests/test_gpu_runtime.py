"""Runtime behaviour on the GPU: checkpointed long runs through the range
API, the host-side wait limit of perm_last_status (no GPU fault involved: a
long but finite launch is simply waited on with a short limit), and a range
split across two streams."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1904_06229_gb300 import longrun as L
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_checkpointed_run_matches_single_call(tmp_path):
    A = W.haar_submatrix(26, 676, 12)
    path = str(tmp_path / "st.json")
    assert L.run(A, path, chunk_codes=1 << 21, max_chunks=5) is None
    got = L.run(A, path, chunk_codes=1 << 21)
    one = P.perm_c128(torch.from_numpy(A).cuda()).cpu().numpy()
    ref = complex(one[0], one[1])
    assert abs(got - ref) <= 1e-12 * abs(ref)


def test_status_wait_limit(monkeypatch):
    A = torch.from_numpy(W.haar_submatrix(40, 1600, 1040)).cuda()
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    P.perm_c128_range(A, 0, 1 << 32, out=out)  # about a second of work
    monkeypatch.setenv("PERM_TIMEOUT_S", "0.001")
    assert P.perm_last_status() == -5  # PERM_ETIMEOUT: gave up waiting, nothing failed
    monkeypatch.delenv("PERM_TIMEOUT_S")
    assert P.perm_last_status() == 0
    assert np.isfinite(out.cpu().numpy()).all()


def test_two_streams_split_one_sum():
    n = 30
    A = torch.from_numpy(W.complex_gaussian(n, 30)).cuda()
    N = 1 << (n - 1)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    o1 = torch.empty(4, dtype=torch.float64, device="cuda")
    o2 = torch.empty(4, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        P.perm_c128_range(A, 0, N // 3, out=o1, stream=s1)
    with torch.cuda.stream(s2):
        P.perm_c128_range(A, N // 3, N - N // 3, out=o2, stream=s2)
    torch.cuda.synchronize()
    p = (o1 + o2).cpu().numpy()
    split = -2 * complex(p[0] + p[1], p[2] + p[3])  # 2 (-1)^(n-1), n even
    full = P.perm_c128(A).cpu().numpy()
    ref = complex(full[0], full[1])
    assert abs(split - ref) <= 1e-12 * abs(ref)

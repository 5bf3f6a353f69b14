"""Runtime behaviour on the GPU: checkpointed long runs through the range
API, the host-side wait limit of perm_last_status (no GPU fault involved: a
long but finite launch is simply waited on with a short limit), a range
split across two streams, reuse after perm_shutdown, and first calls that
return before their work is done."""
import os

import numpy as np
import pytest
import torch

import _tolerance as T
from oracle import oracle as O
from paper_1904_06229_gb300 import longrun as L
from paper_1904_06229_gb300 import perm as P
from paper_1904_06229_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_checkpointed_run_matches_single_call(tmp_path):
    """An interrupted and resumed run in 2^21-code chunks against the oracle
    (the 1e-10 bar) and against one uninterrupted call (the two split the sum
    differently, so they agree to rounding: 1e-11)."""
    A = W.haar_submatrix(26, 676, 12)
    path = str(tmp_path / "st.json")
    assert L.run(A, path, chunk_codes=1 << 21, max_chunks=5) is None
    got = L.run(A, path, chunk_codes=1 << 21)
    one = P.perm_c128(torch.from_numpy(A).cuda()).cpu().numpy()
    single = complex(one[0], one[1])
    re, im, asum = O.per(A)
    T.check(got, complex(float(re), float(im)), float(asum), 26, T.U_DF, "checkpointed n=26")
    assert abs(got - single) <= 1e-11 * abs(single)


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


def test_shutdown_then_reuse():
    """perm_shutdown frees the per-device status words, cached batch graphs and
    the pool reserve; later calls allocate afresh and give the same results,
    and a non-finite input is still reported afterwards."""
    A = torch.from_numpy(W.complex_gaussian(12, 5)).cuda()
    before = P.perm_c128(A).cpu()
    mats = [torch.from_numpy(W.complex_gaussian(n, 40 + n)).cuda() for n in (8, 11, 13)]
    b_before = P.perm_batch(mats).cpu()
    torch.cuda.synchronize()
    P.perm_shutdown()
    P.perm_shutdown()  # twice is fine
    assert torch.equal(P.perm_c128(A).cpu(), before)
    assert torch.equal(P.perm_batch(mats).cpu(), b_before)
    assert P.perm_last_status() == 0
    bad = A.clone()
    bad[3, 4] = complex(float("nan"), 0.0)
    P.perm_c128(bad)
    assert P.STATUS[P.perm_last_status()] == "PERM_ENONFINITE"
    assert P.perm_last_status() == 0


def test_first_calls_return_before_the_work_finishes():
    """Compute calls are asynchronous, the first ones in a process included.
    CUDA loads kernels lazily and a load waits for the device to go idle, so
    the library loads all of its kernels when it first meets a device; a
    second call made while the first one's walk is still running (here a
    modular walk behind an n = 37 FP64 walk of about 5 s) must not wait for
    it."""
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = (
        "import time, torch\n"
        "from paper_1904_06229_gb300 import perm as P, workloads as W\n"
        "A = torch.from_numpy(W.complex_gaussian(37, 7)).cuda()\n"
        "B = torch.from_numpy(W.zero_one(24, 6)).cuda()\n"
        "pr = P.perm_default_primes()\n"
        "torch.cuda.synchronize()\n"
        "t0 = time.perf_counter(); P.perm_c128(A); t1 = time.perf_counter()\n"
        "P.perm_mod01(B, pr); t2 = time.perf_counter()\n"
        "torch.cuda.synchronize(); t3 = time.perf_counter()\n"
        "print(t1 - t0, t2 - t1, t3 - t0)\n"
    )
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, cwd=root, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    first, second, total = map(float, r.stdout.split()[-3:])
    print(f"first call {first:.3f} s, second call {second:.3f} s, all work {total:.3f} s")
    assert total > 2.0
    assert second < 0.25 * total
    assert first + second < 0.5 * total


@pytest.mark.parametrize("stage", ["launch", "finalize"])
def test_injected_failure_then_resume(tmp_path, monkeypatch, stage):
    """PERM_FAULT makes the third range call of a checkpointed run fail on the
    host (no device fault); the run stops with PermError, its checkpoint holds
    the two finished chunks, and resuming gives the uninterrupted result."""
    A = W.haar_submatrix(22, 484, 31)
    ref = L.run(A, str(tmp_path / "ref.json"), chunk_codes=1 << 17)
    path = str(tmp_path / "st.json")
    monkeypatch.setenv("PERM_FAULT", f"{stage}:3")
    with pytest.raises(P.PermError) as e:
        L.run(A, path, chunk_codes=1 << 17)
    assert e.value.code == -3
    assert L.load_state(path)["next"] == 2 << 17
    monkeypatch.delenv("PERM_FAULT")
    assert P.perm_last_status() == 0
    assert L.run(A, path, chunk_codes=1 << 17) == ref

"""Checkpoint / resume of long permanents, with failures injected on the host:
a range call that raises mid-run, then a resume from the state file.  The
per-range partials come from the oracle here (no GPU)."""
import json

import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_06229_gb300 import longrun as L
from paper_1904_06229_gb300 import workloads as W


def oracle_range(A, first, count):
    g = O.glynn_partial(A, first, count)
    re, im = float(g[0]), float(g[1])
    return [re, float(g[0] - np.longdouble(re)), im, float(g[1] - np.longdouble(im))]


def test_uninterrupted_matches_oracle(tmp_path):
    A = W.complex_gaussian(12, 3)
    got = L.run(A, str(tmp_path / "st.json"), chunk_codes=300, range_fn=oracle_range)
    r = O.per(A)
    ref = complex(float(r[0]), float(r[1]))
    assert abs(got - ref) <= 1e-14 * abs(ref)


def test_crash_and_resume(tmp_path):
    A = W.haar_submatrix(11, 121, 4)
    path = str(tmp_path / "st.json")
    calls = {"n": 0}

    def flaky(A_, first, count):
        calls["n"] += 1
        if calls["n"] == 4:
            raise RuntimeError("injected failure")
        return oracle_range(A_, first, count)

    with pytest.raises(RuntimeError):
        L.run(A, path, chunk_codes=100, range_fn=flaky)
    st = json.load(open(path))
    assert st["next"] == 300  # three chunks were recorded before the failure
    got = L.run(A, path, chunk_codes=100, range_fn=oracle_range)
    whole = L.run(A, str(tmp_path / "b.json"), chunk_codes=100, range_fn=oracle_range)
    assert got == whole  # same chunks, same order: bit-identical


def test_stop_and_continue(tmp_path):
    A = W.complex_gaussian(10, 8)
    path = str(tmp_path / "st.json")
    assert L.run(A, path, chunk_codes=64, range_fn=oracle_range, max_chunks=3) is None
    assert json.load(open(path))["next"] == 192
    got = L.run(A, path, chunk_codes=64, range_fn=oracle_range)
    r = O.per(A)
    assert abs(got - complex(float(r[0]), float(r[1]))) <= 1e-14 * abs(complex(float(r[0]), float(r[1])))


def test_refuses_foreign_checkpoint(tmp_path):
    path = str(tmp_path / "st.json")
    L.run(W.complex_gaussian(6, 1), path, chunk_codes=8, range_fn=oracle_range, max_chunks=1)
    with pytest.raises(ValueError):
        L.run(W.complex_gaussian(6, 2), path, chunk_codes=8, range_fn=oracle_range)
    with pytest.raises(ValueError):
        L.run(W.complex_gaussian(6, 1), path, chunk_codes=16, range_fn=oracle_range)

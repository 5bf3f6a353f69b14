"""The batch tuning table's host-side get/set and its JSON file keyed by GPU
name (no device needed: the table is host memory)."""
import json

import pytest

from paper_1904_06229_gb300 import perm as P


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_06229_gb300 import build

    build.build()
    P.load()


def test_get_set_round_trip():
    dev = 7  # any device index: no CUDA call is made
    assert P.perm_batch_tuning(dev) == ([0] * 33, [0] * 33)
    L, K = [0] * 33, [0] * 33
    for n in range(4, 33):
        L[n] = 1 << (4 + n % 8)
        K[n] = 1 + n % 4
    assert P.perm_batch_tuning(dev, L, K) == (L, K)
    assert P.perm_batch_tuning(dev) == (L, K)
    assert P.perm_batch_tuning(dev + 1) == ([0] * 33, [0] * 33)  # per device
    P.perm_batch_tuning(dev, [0] * 33, [0] * 33)


@pytest.mark.parametrize("bad", [15, 24, 1 << 25, -16])
def test_set_rejects_bad_lengths(bad):
    dev = 9
    L, K = [0] * 33, [0] * 33
    L[20], K[20] = 256, 2
    P.perm_batch_tuning(dev, L, K)
    M = list(L)
    M[12] = bad
    K2 = list(K)
    K2[12] = 1
    with pytest.raises(P.PermError) as e:
        P.perm_batch_tuning(dev, M, K2)
    assert e.value.code == -1
    assert P.perm_batch_tuning(dev) == (L, K)  # nothing changed
    P.perm_batch_tuning(dev, [0] * 33, [0] * 33)


@pytest.mark.parametrize("kind,L", [(5, 64), (-1, 64), (0, 64), (2, 0)])
def test_set_rejects_bad_kinds(kind, L):
    dev = 10
    Ls, Ks = [0] * 33, [0] * 33
    Ls[14], Ks[14] = L, kind
    with pytest.raises(P.PermError):
        P.perm_batch_tuning(dev, Ls, Ks)
    assert P.perm_batch_tuning(dev) == ([0] * 33, [0] * 33)


def test_argument_errors():
    with pytest.raises(P.PermError):
        P.perm_batch_tuning(64)
    with pytest.raises(ValueError):
        P.perm_batch_tuning(0, [0] * 32, [0] * 32)
    with pytest.raises(ValueError):
        P.perm_batch_tuning(0, [0] * 33)


def test_json_file_keyed_by_name(tmp_path):
    path = str(tmp_path / "tune.json")
    L, K = [0] * 33, [0] * 33
    L[28], K[28] = 512, 2
    P.perm_batch_tuning(3, L, K)
    P.save_batch_tuning(path, device=3, name="GPU A")
    P.perm_batch_tuning(3, [0] * 33, [0] * 33)
    assert P.load_batch_tuning(path, device=3, name="GPU B") is False
    assert P.load_batch_tuning(path, device=3, name="GPU A") is True
    assert P.perm_batch_tuning(3) == (L, K)
    saved = json.load(open(path))["GPU A"]
    assert saved["L"][28] == 512 and saved["kind"][28] == 2
    P.perm_batch_tuning(3, [0] * 33, [0] * 33)


def test_plan_counter_without_device():
    assert P.perm_batch_plans() >= 0

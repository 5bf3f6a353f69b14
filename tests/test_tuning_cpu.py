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
    assert P.perm_batch_tuning(dev) == [0] * 33
    L = [0] * 33
    for n in range(4, 33):
        L[n] = 1 << (4 + n % 8)
    assert P.perm_batch_tuning(dev, L) == L
    assert P.perm_batch_tuning(dev) == L
    assert P.perm_batch_tuning(dev + 1) == [0] * 33  # per device
    P.perm_batch_tuning(dev, [0] * 33)


@pytest.mark.parametrize("bad", [15, 24, 1 << 25, -16])
def test_set_rejects_bad_lengths(bad):
    dev = 9
    L = [0] * 33
    L[20] = 256
    P.perm_batch_tuning(dev, L)
    M = list(L)
    M[12] = bad
    with pytest.raises(P.PermError) as e:
        P.perm_batch_tuning(dev, M)
    assert e.value.code == -1
    assert P.perm_batch_tuning(dev) == L  # nothing changed
    P.perm_batch_tuning(dev, [0] * 33)


def test_argument_errors():
    with pytest.raises(P.PermError):
        P.perm_batch_tuning(64)
    with pytest.raises(ValueError):
        P.perm_batch_tuning(0, [0] * 32)


def test_json_file_keyed_by_name(tmp_path):
    path = str(tmp_path / "tune.json")
    L = [0] * 33
    L[28] = 512
    P.perm_batch_tuning(3, L)
    P.save_batch_tuning(path, device=3, name="GPU A")
    P.perm_batch_tuning(3, [0] * 33)
    assert P.load_batch_tuning(path, device=3, name="GPU B") is False
    assert P.load_batch_tuning(path, device=3, name="GPU A") is True
    assert P.perm_batch_tuning(3) == L
    assert json.load(open(path))["GPU A"][28] == 512
    P.perm_batch_tuning(3, [0] * 33)

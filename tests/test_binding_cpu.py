"""The Python binding's argument checks on the CPU: wrong dtypes, shapes and
buffers are refused before the library is called, and a compute call made
without a device raises PermError(PERM_ECUDA) instead of computing anything
on the host."""
import pytest
import torch

from paper_1904_06229_gb300 import perm as P


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_06229_gb300 import build

    build.build()
    P.load()


def test_dtype_and_shape_checks():
    with pytest.raises(TypeError):
        P.perm_c128(torch.zeros(3, 3, dtype=torch.float64))
    with pytest.raises(TypeError):
        P.perm_f64(torch.zeros(3, 3, dtype=torch.complex128))
    with pytest.raises(ValueError):
        P.perm_c128(torch.zeros(3, 4, dtype=torch.complex128))
    with pytest.raises(ValueError):
        P.perm_f64(torch.zeros(2, 2, 2, dtype=torch.float64))
    with pytest.raises(ValueError):
        P.perm_c128(torch.zeros(3, 3, dtype=torch.complex128), out=torch.empty(1, dtype=torch.float64))


def test_empty_batches_refused():
    with pytest.raises(ValueError):
        P.perm_batch([])
    with pytest.raises(ValueError):
        P.perm_batch_stats([])


def test_batch_type_checks():
    with pytest.raises(TypeError):
        P.perm_batch([torch.zeros(3, 3, dtype=torch.float64)])


def test_no_device_raises_instead_of_computing():
    if torch.cuda.is_available():
        pytest.skip("device present")
    A = torch.eye(4, dtype=torch.complex128)
    with pytest.raises(P.PermError) as e:
        P.perm_c128(A)
    assert e.value.code == -3
    with pytest.raises(P.PermError) as e:
        P.perm_f64(torch.eye(4, dtype=torch.float64))
    assert e.value.code == -3


def test_status_names_cover_the_header():
    assert sorted(P.STATUS) == [-7, -6, -5, -4, -3, -2, -1, 0]
    for code, name in P.STATUS.items():
        assert P.perm_status_string(code).startswith(name)

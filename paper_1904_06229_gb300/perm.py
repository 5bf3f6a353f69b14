"""Python binding of libperm.so (include/perm.h): argument marshalling only.

Each function has the name of the C entry point it calls, takes torch tensors
(CUDA tensors are passed by device pointer, CPU tensors by host pointer: the
library copies host buffers itself) and the current CUDA stream, and raises
`PermError` on a non-zero status.  Nothing here computes any part of a
permanent; without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libperm.so")
PERM_NMAX = 64

STATUS = {
    0: "PERM_OK",
    -1: "PERM_EINVAL",
    -2: "PERM_ENULL",
    -3: "PERM_ECUDA",
    -4: "PERM_ENONFINITE",
    -5: "PERM_ETIMEOUT",
    -6: "PERM_ENOMEM",
    -7: "PERM_EPRIME",
}

# every symbol include/perm.h declares
EXPORTS = [
    "perm_c128",
    "perm_f64",
    "perm_c128_range",
    "perm_f64_range",
    "perm_c128_f32p",
    "perm_f64_f32p",
    "perm_c128_noalloc",
    "perm_c128_repeated",
    "perm_c128_band",
    "perm_c128_sparse",
    "perm_sparse_partition",
    "perm_batch",
    "perm_batch_stats",
    "perm_batch_autotune",
    "perm_batch_tuning",
    "perm_batch_plans",
    "perm_mod01",
    "perm_crt",
    "perm_default_primes",
    "perm_last_status",
    "perm_status_string",
    "perm_fp64_peak",
    "perm_pipe_peak",
    "perm_shutdown",
]


class PermError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")
        self.code = code


_lib = None
_lock = threading.Lock()


def load(path: Optional[str] = None):
    """Load libperm.so (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libperm.so is not built ({p}); run `python -m paper_1904_06229_gb300.build`")
        lib = ctypes.CDLL(p)
        vp, i, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
        for name, args in {
            "perm_c128": [vp, i, vp, vp],
            "perm_f64": [vp, i, vp, vp],
            "perm_c128_range": [vp, i, u64, u64, vp, vp],
            "perm_f64_range": [vp, i, u64, u64, vp, vp],
            "perm_c128_f32p": [vp, i, vp, vp],
            "perm_f64_f32p": [vp, i, vp, vp],
            "perm_c128_noalloc": [vp, i, vp, vp],
            "perm_c128_repeated": [vp, vp, i, i, vp, vp],
            "perm_c128_band": [vp, i, i, i, vp, vp],
            "perm_c128_sparse": [vp, i, vp, vp],
            "perm_sparse_partition": [vp, i, vp, vp],
            "perm_batch": [vp, vp, i, vp, vp],
            "perm_batch_stats": [vp, vp, i, vp, vp, vp],
            "perm_batch_autotune": [i, i],
            "perm_batch_tuning": [i, vp, vp, i],
            "perm_batch_plans": [vp],
            "perm_mod01": [vp, i, vp, vp, vp],
            "perm_crt": [vp, vp, i, vp],
            "perm_default_primes": [vp],
            "perm_last_status": [vp],
            "perm_status_string": [i],
            "perm_fp64_peak": [vp],
            "perm_pipe_peak": [i, vp],
            "perm_shutdown": [],
        }.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.perm_status_string.restype = ctypes.c_char_p
        lib.perm_shutdown.restype = None
        _lib = lib
        return lib


def _check(rc: int, where: str):
    if rc != 0:
        raise PermError(rc, where)


def _stream(t: Optional[torch.Tensor], stream) -> Optional[int]:
    if stream is not None:
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    if t is not None and t.is_cuda:
        return int(torch.cuda.current_stream(t.device).cuda_stream)
    if torch.cuda.is_available():
        return int(torch.cuda.current_stream().cuda_stream)
    return None


def _square(A: torch.Tensor) -> int:
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square matrix")
    return int(A.shape[0])


def _dptr(t: torch.Tensor) -> int:
    return int(t.data_ptr())


def _c128(A: torch.Tensor) -> torch.Tensor:
    if A.dtype != torch.complex128:
        raise TypeError("complex128 matrix expected")
    return A.contiguous()


def _f64(A: torch.Tensor) -> torch.Tensor:
    if A.dtype != torch.float64:
        raise TypeError("float64 matrix expected")
    return A.contiguous()


def _out(out: Optional[torch.Tensor], n: int, like: torch.Tensor, dtype=torch.float64) -> torch.Tensor:
    if out is None:
        out = torch.empty(n, dtype=dtype, device=like.device)
    if out.numel() < n or not out.is_contiguous():
        raise ValueError("output buffer too small or not contiguous")
    return out


def perm_c128(A: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """per(A) of a complex128 n x n tensor -> float64 tensor [re, im]."""
    A = _c128(A)
    n = _square(A)
    out = _out(out, 2, A)
    _check(load().perm_c128(_dptr(A), n, _dptr(out), _stream(A, stream)), "perm_c128")
    return out


def perm_f64(A: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """per(A) of a float64 n x n tensor -> float64 tensor [value]."""
    A = _f64(A)
    n = _square(A)
    out = _out(out, 1, A)
    _check(load().perm_f64(_dptr(A), n, _dptr(out), _stream(A, stream)), "perm_f64")
    return out


def perm_c128_range(A: torch.Tensor, first: int, count: int, out: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
    """Unscaled Gray-code partial over [first, first+count) -> [re_hi, re_lo, im_hi, im_lo]."""
    A = _c128(A)
    n = _square(A)
    out = _out(out, 4, A)
    _check(load().perm_c128_range(_dptr(A), n, int(first), int(count), _dptr(out), _stream(A, stream)),
           "perm_c128_range")
    return out


def perm_f64_range(A: torch.Tensor, first: int, count: int, out: Optional[torch.Tensor] = None,
                   stream=None) -> torch.Tensor:
    A = _f64(A)
    n = _square(A)
    out = _out(out, 2, A)
    _check(load().perm_f64_range(_dptr(A), n, int(first), int(count), _dptr(out), _stream(A, stream)),
           "perm_f64_range")
    return out


def perm_c128_f32p(A: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    A = _c128(A)
    n = _square(A)
    out = _out(out, 2, A)
    _check(load().perm_c128_f32p(_dptr(A), n, _dptr(out), _stream(A, stream)), "perm_c128_f32p")
    return out


def perm_f64_f32p(A: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    A = _f64(A)
    n = _square(A)
    out = _out(out, 1, A)
    _check(load().perm_f64_f32p(_dptr(A), n, _dptr(out), _stream(A, stream)), "perm_f64_f32p")
    return out


def perm_c128_noalloc(A: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    """perm_c128 without any device allocation: A and out must be CUDA
    tensors (complex128 n x n, float64 (2,)).  Calls that overlap on the GPU
    share one scratch array and must be serialised."""
    A = _c128(A)
    n = _square(A)
    _check(load().perm_c128_noalloc(_dptr(A), n, _dptr(out), _stream(A, stream)), "perm_c128_noalloc")
    return out


def perm_c128_repeated(Cbar: torch.Tensor, mult: Sequence[int], out: Optional[torch.Tensor] = None,
                       stream=None) -> torch.Tensor:
    """Eq.(ryser2): permanent of the matrix whose distinct columns are the
    columns of the complex128 n x R tensor `Cbar`, column k repeated mult[k]
    times -> float64 tensor [re, im]."""
    if Cbar.dtype != torch.complex128 or Cbar.dim() != 2:
        raise TypeError("complex128 n x R tensor expected")
    Cbar = Cbar.contiguous()
    n, R = int(Cbar.shape[0]), int(Cbar.shape[1])
    if len(mult) != R:
        raise ValueError("one multiplicity per distinct column")
    m = (ctypes.c_int * R)(*[int(v) for v in mult])
    out = _out(out, 2, Cbar)
    _check(load().perm_c128_repeated(_dptr(Cbar), ctypes.addressof(m), R, n, _dptr(out), _stream(Cbar, stream)),
           "perm_c128_repeated")
    return out


def perm_c128_band(A: torch.Tensor, k: int, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """App. C band permanent of a complex128 n x n tensor, or of each matrix
    of a (count, n, n) tensor, with half-bandwidth k -> float64 (count, 2)."""
    if A.dtype != torch.complex128:
        raise TypeError("complex128 matrices expected")
    A = A.contiguous()
    if A.dim() == 2:
        A = A.unsqueeze(0)
    if A.dim() != 3 or A.shape[1] != A.shape[2]:
        raise ValueError("(count, n, n) or (n, n) expected")
    count, n = int(A.shape[0]), int(A.shape[1])
    if out is None:
        out = torch.empty((count, 2), dtype=torch.float64, device=A.device)
    _check(load().perm_c128_band(_dptr(A), n, int(k), count, _dptr(out), _stream(A, stream)), "perm_c128_band")
    return out


def perm_c128_sparse(A: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """App. B sparse permanent of a complex128 n x n tensor -> float64 [re, im]."""
    A = _c128(A)
    n = _square(A)
    out = _out(out, 2, A)
    _check(load().perm_c128_sparse(_dptr(A), n, _dptr(out), _stream(A, stream)), "perm_c128_sparse")
    return out


def perm_sparse_partition(A) -> tuple:
    """(block list, number of sets) of the partition perm_c128_sparse uses;
    A is a host complex128 n x n array or tensor."""
    import numpy as np

    a = np.ascontiguousarray(np.asarray(A.cpu() if isinstance(A, torch.Tensor) else A, dtype=np.complex128))
    n = a.shape[0]
    block = (ctypes.c_int * n)()
    count = ctypes.c_uint64(0)
    _check(load().perm_sparse_partition(a.ctypes.data, n, ctypes.addressof(block), ctypes.addressof(count)),
           "perm_sparse_partition")
    return [int(v) for v in block], int(count.value)


def _launch_stream(dev, stream):
    """(raw handle, torch stream) of the stream a call runs on."""
    if stream is None:
        st = torch.cuda.current_stream(dev)
    elif hasattr(stream, "cuda_stream"):
        st = stream
    else:
        st = torch.cuda.ExternalStream(int(stream), device=dev)
    return int(st.cuda_stream), st


def _batch_args(mats, out, ptrs, stream):
    """Orders, pointer tensor, output and launch stream of a batch call.  A
    pointer array or output made here is created on the current stream; when
    the call runs on another stream, that stream first waits for the current
    one (the copy of the pointers, the caller's matrices) and the temporaries
    are recorded on it, so the caching allocator cannot hand their memory to
    other work before the batch has read them."""
    count = len(mats)
    if count == 0:
        raise ValueError("empty batch")
    dev = mats[0].device
    ns = (ctypes.c_int * count)(*[_square(m) for m in mats])
    for m in mats:
        if m.dtype != torch.complex128 or not m.is_contiguous() or m.device != dev:
            raise TypeError("contiguous complex128 matrices on one device expected")
    made = []
    if ptrs is None:
        ptrs = torch.tensor([m.data_ptr() for m in mats], dtype=torch.int64).to(dev)
        made.append(ptrs)
    if out is None:
        out = torch.empty((count, 2), dtype=torch.float64, device=dev)
        made.append(out)
    raw, st = _launch_stream(dev, stream)
    cur = torch.cuda.current_stream(dev)
    if st.cuda_stream != cur.cuda_stream:
        st.wait_stream(cur)
        for t in made:
            t.record_stream(st)
    return ns, ptrs, out, raw, st, made


def perm_batch(mats: Sequence[torch.Tensor], out: Optional[torch.Tensor] = None, stream=None,
               ptrs: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Permanents of a list of complex128 CUDA matrices -> (count, 2) float64.

    `ptrs` may pass a prebuilt device int64 tensor of the matrices' addresses."""
    ns, ptrs, out, raw, _, _ = _batch_args(mats, out, ptrs, stream)
    _check(load().perm_batch(_dptr(ptrs), ctypes.addressof(ns), len(mats), _dptr(out), raw), "perm_batch")
    return out


PERM_STATS_STRIDE = 103


def perm_batch_stats(mats: Sequence[torch.Tensor], out: Optional[torch.Tensor] = None,
                     stats: Optional[torch.Tensor] = None, stream=None, ptrs: Optional[torch.Tensor] = None):
    """perm_batch plus the per-order statistics of X = |per| / sqrt(n!) ->
    (out (count, 2), stats (33, PERM_STATS_STRIDE)); see include/perm.h."""
    ns, ptrs, out, raw, st, _ = _batch_args(mats, out, ptrs, stream)
    if stats is None:
        stats = torch.empty((33, PERM_STATS_STRIDE), dtype=torch.float64, device=mats[0].device)
        if st.cuda_stream != torch.cuda.current_stream(mats[0].device).cuda_stream:
            stats.record_stream(st)
    _check(load().perm_batch_stats(_dptr(ptrs), ctypes.addressof(ns), len(mats), _dptr(out), _dptr(stats), raw),
           "perm_batch_stats")
    return out, stats


def perm_batch_plans() -> int:
    """Number of batch plans (graphs) this process has built so far."""
    v = ctypes.c_int(0)
    _check(load().perm_batch_plans(ctypes.addressof(v)), "perm_batch_plans")
    return int(v.value)


def perm_batch_autotune(n_lo: int, n_hi: int) -> None:
    _check(load().perm_batch_autotune(int(n_lo), int(n_hi)), "perm_batch_autotune")


BATCH_KINDS = {"warp": 1, "cta": 2, "cta3": 3, "cta256": 4}


def perm_batch_tuning(device: int, L: Optional[Sequence[int]] = None, kind: Optional[Sequence[int]] = None):
    """Read the batch tuning table of `device` (L and kind None), or replace it
    (33 ints each: for order n, L[n] codes per thread and kind[n] the kernel,
    1 warp per item, 2 block of 128 threads per item, 3 the same with three
    blocks per SM, 4 block of 256 threads per item; 0 = untuned); returns the
    table in force afterwards as (L, kind)."""
    buf = (ctypes.c_int * 33)()
    kbuf = (ctypes.c_int * 33)()
    if L is not None or kind is not None:
        if L is None or kind is None or len(L) != 33 or len(kind) != 33:
            raise ValueError("33 entries expected in both L and kind (orders 0..32)")
        for k in range(33):
            buf[k] = int(L[k])
            kbuf[k] = int(kind[k])
        _check(load().perm_batch_tuning(int(device), ctypes.addressof(buf), ctypes.addressof(kbuf), 1),
               "perm_batch_tuning")
    _check(load().perm_batch_tuning(int(device), ctypes.addressof(buf), ctypes.addressof(kbuf), 0),
           "perm_batch_tuning")
    return [int(v) for v in buf], [int(v) for v in kbuf]


def save_batch_tuning(path: str, device: int = 0, name: Optional[str] = None) -> None:
    """Add this device's batch tuning table to the JSON file at `path`, keyed
    by the GPU's name (torch.cuda.get_device_name unless `name` is given)."""
    import json

    key = name if name is not None else torch.cuda.get_device_name(device)
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    L, kind = perm_batch_tuning(device)
    data[key] = {"L": L, "kind": kind}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load_batch_tuning(path: str, device: int = 0, name: Optional[str] = None) -> bool:
    """Load the table saved for this GPU's name into `device`; False when the
    file has none for it."""
    import json

    key = name if name is not None else torch.cuda.get_device_name(device)
    if not os.path.exists(path):
        return False
    with open(path) as f:
        data = json.load(f)
    if key not in data:
        return False
    perm_batch_tuning(device, data[key]["L"], data[key]["kind"])
    return True


def perm_default_primes() -> list:
    buf = (ctypes.c_uint64 * 4)()
    _check(load().perm_default_primes(ctypes.addressof(buf)), "perm_default_primes")
    return [int(v) for v in buf]


def perm_mod01(A: torch.Tensor, primes: Optional[Sequence[int]] = None, residues: Optional[torch.Tensor] = None,
               stream=None) -> torch.Tensor:
    """per(A) mod each of four primes for an int8 n x n tensor -> int64 tensor (4,)."""
    if A.dtype != torch.int8:
        raise TypeError("int8 matrix expected")
    A = A.contiguous()
    n = _square(A)
    if primes is None:
        primes = perm_default_primes()
    pr = (ctypes.c_uint64 * 4)(*[int(p) for p in primes])
    residues = _out(residues, 4, A, dtype=torch.int64)
    _check(load().perm_mod01(_dptr(A), n, ctypes.addressof(pr), _dptr(residues), _stream(A, stream)), "perm_mod01")
    return residues


def perm_crt(residues: Sequence[int], primes: Sequence[int]) -> int:
    """Signed integer with the given residues (|x| <= P/2), via the library's host CRT."""
    k = len(primes)
    r = (ctypes.c_uint64 * k)(*[int(v) for v in residues])
    p = (ctypes.c_uint64 * k)(*[int(v) for v in primes])
    out = (ctypes.c_uint64 * 4)()
    _check(load().perm_crt(ctypes.addressof(r), ctypes.addressof(p), k, ctypes.addressof(out)), "perm_crt")
    v = sum(int(out[i]) << (64 * i) for i in range(4))
    return v - (1 << 256) if v >> 255 else v


def perm_last_status(stream=None) -> int:
    """Wait for the stream and return (and clear) the device-side status code."""
    return int(load().perm_last_status(_stream(None, stream)))


def perm_status_string(code: int) -> str:
    return load().perm_status_string(int(code)).decode()


def perm_fp64_peak() -> float:
    """Measured FP64 DFMA rate of the current device, in Gop/s (lane DFMAs)."""
    v = ctypes.c_double(0.0)
    _check(load().perm_fp64_peak(ctypes.addressof(v)), "perm_fp64_peak")
    return float(v.value)


PIPES = {"dfma": 0, "ffma": 1, "ffma2": 2, "imad": 3, "alu": 4, "issue": 5}


def perm_pipe_peak(pipe: str) -> float:
    """Measured throughput of one instruction kind (see PIPES) on the current
    device, in G lane instructions/s."""
    v = ctypes.c_double(0.0)
    _check(load().perm_pipe_peak(PIPES[pipe], ctypes.addressof(v)), "perm_pipe_peak")
    return float(v.value)


def perm_shutdown() -> None:
    load().perm_shutdown()

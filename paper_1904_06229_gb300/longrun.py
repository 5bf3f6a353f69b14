"""Long permanents in bounded, checkpointed chunks.

A permanent of order n is a sum over 2^(n-1) Gray codes; at n = 48 on one
GB300 that is many hours.  `run` walks the code range in chunks with
`perm_c128_range` (or `perm_f64_range`), adds each chunk's double-double
partial on the host in chunk order, and after every chunk writes the state --
the next code index and the running partial -- to a JSON file (written to a
temporary name and renamed, so a crash never leaves a torn file).  Calling
`run` again with the same file resumes at the recorded index; the result is
the same as an uninterrupted run because the chunk boundaries and the order
of the additions are the same.

The state file also records the matrix's SHA-256 and the chunk size, and a
resume with a different matrix or chunk size is refused.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, Optional

import numpy as np

from .multirank import dd_add

RangeFn = Callable[[np.ndarray, int, int], list]


def _digest(A: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(A).tobytes()).hexdigest()


def load_state(path: str) -> Optional[dict]:
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def _save_state(path: str, st: dict) -> None:
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(st, f)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def gpu_range_fn(complex_input: bool = True) -> RangeFn:
    """Range function backed by the CUDA library (perm_c128_range / perm_f64_range)."""
    import torch

    from . import perm as P

    def fn(A: np.ndarray, first: int, count: int) -> list:
        dev = torch.device("cuda", torch.cuda.current_device())
        if complex_input:
            t = torch.from_numpy(np.ascontiguousarray(A.astype(np.complex128))).to(dev)
            o = P.perm_c128_range(t, first, count).cpu().tolist()
        else:
            t = torch.from_numpy(np.ascontiguousarray(A.astype(np.float64))).to(dev)
            hi, lo = P.perm_f64_range(t, first, count).cpu().tolist()
            o = [hi, lo, 0.0, 0.0]
        return o

    return fn


def run(A: np.ndarray, path: str, chunk_codes: int = 1 << 34, range_fn: Optional[RangeFn] = None,
        max_chunks: Optional[int] = None) -> Optional[complex]:
    """Compute per(A) in checkpointed chunks.  Returns the permanent when the
    whole range is done, or None if `max_chunks` stopped it early (the state
    file then holds the progress)."""
    A = np.asarray(A)
    n = A.shape[0]
    total = 1 << (n - 1)
    if range_fn is None:
        range_fn = gpu_range_fn(np.iscomplexobj(A))
    digest = _digest(A)
    st = load_state(path)
    if st is None:
        st = {"n": n, "sha256": digest, "chunk": int(chunk_codes), "next": 0, "re": [0.0, 0.0], "im": [0.0, 0.0]}
    elif st["sha256"] != digest or st["chunk"] != int(chunk_codes) or st["n"] != n:
        raise ValueError("checkpoint belongs to another matrix or chunk size")
    done_chunks = 0
    while st["next"] < total:
        if max_chunks is not None and done_chunks >= max_chunks:
            return None
        first = st["next"]
        count = min(int(chunk_codes), total - first)
        p = range_fn(A, first, count)
        st["re"] = list(dd_add(tuple(st["re"]), (float(p[0]), float(p[1]))))
        st["im"] = list(dd_add(tuple(st["im"]), (float(p[2]), float(p[3]))))
        st["next"] = first + count
        _save_state(path, st)
        done_chunks += 1
    s = 2.0 if (n - 1) % 2 == 0 else -2.0
    return complex(s * (st["re"][0] + st["re"][1]), s * (st["im"][0] + st["im"][1]))

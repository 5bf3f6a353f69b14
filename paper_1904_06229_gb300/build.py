"""Build libperm.so for sm_103a with nvcc (no cmake, no torch extension
machinery): each translation unit is compiled in parallel, then linked into
paper_1904_06229_gb300/_build/libperm.so.  Objects are rebuilt only when a
source or header is newer.  The CUDA runtime is linked statically, so the
library needs only the driver at run time.

    python -m paper_1904_06229_gb300.build
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libperm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = [
    "walk_c128_f64_lo.cu",
    "walk_c128_f64_hi.cu",
    "walk_r64_f64.cu",
    "walk_c128_f32.cu",
    "walk_r64_f32.cu",
    "walk_fx_c128_f64_lo.cu",
    "walk_fx_c128_f64_hi.cu",
    "walk_fx_r64_f64.cu",
    "walk_fx_c128_f32.cu",
    "walk_fx_r64_f32.cu",
    "walk_df_c128.cu",
    "walk_xp_c128_lo.cu",
    "walk_xp_c128_hi.cu",
    "walk_pdf_c128_lo.cu",
    "walk_pdf_c128_hi.cu",
    "walk_pdf_r64_lo.cu",
    "walk_pdf_r64_hi.cu",
    "glynn_mod.cu",
    "mod_lo.cu",
    "mod_mid.cu",
    "mod_hi.cu",
    "ryser2.cu",
    "band.cu",
    "sparse.cu",
    "batch.cu",
    "batch_cta2.cu",
    "batch_cta3.cu",
    "batch_cta256.cu",
    "perm_abi.cu",
    "peak.cu",
    "noalloc.cu",
    "host_modular.cpp",
]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libperm.so")
    return cand


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(obj: str, src: str, hdr_mtime: float) -> bool:
    if not os.path.exists(obj):
        return True
    m = os.path.getmtime(obj)
    return m < os.path.getmtime(src) or m < hdr_mtime


def build(verbose: bool = False, jobs: int = 0) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    hdr_mtime = max([os.path.getmtime(h) for h in _headers()] + [0.0])
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
    objs, todo = [], []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT_DIR, os.path.splitext(s)[0] + ".o")
        objs.append(obj)
        if _stale(obj, src, hdr_mtime):
            todo.append((src, obj))

    def compile_one(item):
        src, obj = item
        tmp = obj + f".{os.getpid()}.tmp.o"
        cmd = [nvcc] + flags + ["-c", src, "-o", tmp]
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{res.stderr[-4000:]}")
        os.replace(tmp, obj)
        return src

    if todo:
        workers = jobs or min(len(todo), os.cpu_count() or 4)
        with ThreadPoolExecutor(max_workers=workers) as ex:
            for _ in ex.map(compile_one, todo):
                pass
    if todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stderr[-4000:]}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))

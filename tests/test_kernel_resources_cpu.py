"""Register and spill budget of the hot kernels, read from ptxas's resource
report at compile time (no GPU): the measured rates depend on the default
packed walk at n = 40 and 48, the block-per-item batch kernel, the warp batch
kernel and the modular kernel at the benchmarked orders staying (nearly) free
of register spills: none for the walks, the block batch kernel and the
modular kernel, at most 8 bytes for the warp batch kernel (which holds every
order up to 32 in one kernel)."""
import os
import re
import shutil
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_06229_gb300", "csrc")
INC = os.path.join(ROOT, "include")

# (source file, mangled-name fragment of the kernel, what it is, spill bytes allowed)
CASES = [
    ("walk_pdf_c128_hi.cu", "k_walk_xpILi40ELb0E", "n = 40 packed walk (bench)", 0),
    ("walk_pdf_c128_hi.cu", "k_walk_xpILi48ELb0E", "n = 48 packed walk", 0),
    ("batch_cta2.cu", "k_batch_ctaILi2E", "block-per-item batch kernel", 0),
    ("walk_fx_c128_f64_hi.cu", "k_walk_fxILi40ELb1ELi0E", "n = 40 fixed-point walk", 0),
    ("walk_fx_c128_f64_hi.cu", "k_walk_fxILi36ELb1ELi0E", "n = 36 complex walk", 0),
    ("batch.cu", "k_batchILi1E", "batch kernel, fixed-point rows", 8),
    ("mod_lo.cu", "k_modILi30E", "exact 0-1, n = 30", 0),
    ("mod_mid.cu", "k_modILi36E", "exact 0-1, n = 36", 0),
]


def _nvcc():
    return shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def _report(src):
    from paper_1904_06229_gb300 import build

    with tempfile.TemporaryDirectory() as d:
        cmd = [_nvcc()] + build.ARCH + ["-O3", "-std=c++17", "-I", CSRC, "-I", INC, "-Xptxas", "-v", "-c",
                                        os.path.join(CSRC, src), "-o", os.path.join(d, "o.o")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        return r.stderr


@pytest.fixture(scope="module")
def reports():
    if not os.path.exists(_nvcc()):
        pytest.skip("nvcc not available")
    srcs = sorted({c[0] for c in CASES})
    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        return dict(zip(srcs, ex.map(_report, srcs)))


@pytest.mark.parametrize("src,frag,what,allowed", CASES)
def test_spill_budget(reports, src, frag, what, allowed):
    text = reports[src]
    m = re.search(r"Function properties for \S*" + re.escape(frag) + r"\S*\n\s*(\d+) bytes stack frame, (\d+) bytes "
                  r"spill stores, (\d+) bytes spill loads", text)
    assert m, f"no resource report for {what}"
    assert int(m.group(2)) <= allowed and int(m.group(3)) <= allowed, f"{what} spills: {m.group(0)}"

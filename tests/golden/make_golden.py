"""Write tests/golden/configs.json: oracle values of the full-size seeded
configurations whose permanents the CPU oracle can finish in about an hour.

This script imports only the oracle (`oracle/`) and the seeded input
generators (`paper_1904_06229_gb300/workloads.py`, which holds no arithmetic
of the method); no value in the file comes from the CUDA library.  Each entry
stores the matrix itself (0-1 and +-1 entries as digit strings, floats as
exact hex), so a test compares against the very matrix the value belongs to
and checks separately that the generator still produces it.

Configurations (sizes and seeds of the paper-shaped workloads):
  zero_one_n36_seed7   0-1 entries, density 1/2, n = 36: Sec. 2.B (exact
                       permanents of 0-1 matrices), 2^35 codes of the exact
                       512-bit App. A walk (about an hour on 8 cores).
  zero_one_n30_seed6   the same at n = 30 (2^29 codes).
  pm1_n30_seed5        +-1 Bernoulli(1/2), n = 30 (Sec. 5), exact.
  real_gaussian_n32_seed4  real N(0,1), n = 32, long double App. A walk with
                       Neumaier-compensated summation; also its sum of term
                       magnitudes (condition number of the sum).

Usage: python tests/golden/make_golden.py [--only NAME ...] [--threads T]
Entries not named keep their stored values.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(os.path.dirname(_HERE))
sys.path.insert(0, _ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1904_06229_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(_HERE, "configs.json")


def _int_rows(A) -> list[str]:
    """Integer matrix rows as strings of signed digits ("0", "1", "-1" joined by spaces)."""
    return [" ".join(str(int(v)) for v in row) for row in np.asarray(A)]


def _hex_rows(A) -> list[str]:
    return [" ".join(float(v).hex() for v in row) for row in np.asarray(A, dtype=np.float64)]


def _ld(x) -> str:
    return np.format_float_scientific(np.longdouble(x), precision=21, unique=False)


def make_exact(name: str, A, source: str, threads: int) -> dict:
    t0 = time.time()
    v = O.per_exact(A, parts=4096, threads=threads)
    dt = time.time() - t0
    e = {"name": name, "kind": "exact", "n": int(A.shape[0]), "matrix": _int_rows(A), "per": str(v),
         "per_bits": v.bit_length() if v else 0, "oracle": "oracle.per_exact (512-bit App. A walk, v = 2w)",
         "seconds": round(dt, 1), "source": source}
    if A.shape[0] <= 32:
        # sum of the term magnitudes (long double walk): the condition number
        # that the floating-point bounds of the tests use
        e["abs_sum"] = _ld(O.per(A.astype(np.float64), threads=threads)[2])
    return e


def make_real(name: str, A, source: str, threads: int) -> dict:
    t0 = time.time()
    re, im, asum = O.per(A, threads=threads)
    dt = time.time() - t0
    return {"name": name, "kind": "long_double", "n": int(A.shape[0]), "matrix": _hex_rows(A), "per": _ld(re),
            "per_im": _ld(im), "abs_sum": _ld(asum), "long_double_digits": O.long_double_digits(),
            "oracle": "oracle.per (App. A walk, long double, Neumaier-compensated)", "seconds": round(dt, 1),
            "source": source}


CONFIGS = {
    "zero_one_n30_seed6": (lambda: W.zero_one(30, 6), make_exact,
                           "workloads.zero_one(30, 6): 0-1 density 1/2 (Sec. 2.B exact 0-1 permanents)"),
    "pm1_n30_seed5": (lambda: W.bernoulli_pm1(30, 5), make_exact,
                      "workloads.bernoulli_pm1(30, 5): +-1 Bernoulli(1/2) (Sec. 5)"),
    "real_gaussian_n32_seed4": (lambda: W.real_gaussian(32, 4), make_real,
                                "workloads.real_gaussian(32, 4): real N(0,1) (precision study)"),
    "zero_one_n36_seed7": (lambda: W.zero_one(36, 7), make_exact,
                           "workloads.zero_one(36, 7): 0-1 density 1/2 (Sec. 2.B exact 0-1 permanents)"),
}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    data = {"_about": ("Oracle values of full-size seeded configurations, written by tests/golden/make_golden.py "
                       "(oracle/ and workloads.py only; nothing from the CUDA library)."), "cases": {}}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    names = args.only if args.only else list(CONFIGS)
    for name in names:
        gen, fn, src = CONFIGS[name]
        A = gen()
        entry = fn(name, A, src, args.threads)
        entry["host"] = f"{platform.machine()}, {os.cpu_count()} cores"
        data["cases"][name] = entry
        with open(OUT + ".tmp", "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")
        os.replace(OUT + ".tmp", OUT)
        print(name, entry["per"], f"{entry['seconds']} s", flush=True)


if __name__ == "__main__":
    main()

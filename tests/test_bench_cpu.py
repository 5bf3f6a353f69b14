"""The bench's reference arm (the CPU oracle timed on the host cores) and its
argument checks, on the CPU: one JSON line with the contract's keys; the
roofline's operation counts."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          cwd=ROOT, timeout=timeout)


def test_reference_arm_json_line():
    r = _run("--impl", "reference", "--steps", "2", "--warmup", "3", "--reference-step-seconds", "0.2")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["unit"] == "terms/s" and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_warmup_below_three_is_refused():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "2", timeout=120)
    assert r.returncode != 0
    assert "warmup" in (r.stderr + r.stdout)


def test_fp32_operation_counts_of_the_roofline():
    """The roofline's FP32 operations per code, hand-counted from the default
    walk's arithmetic: per row pair and step two 11-operation packed
    double-float adds (22 packed = 44 lane operations), NP - 1 packed complex
    products of 32 (64 lane operations), a 4-operation packed renormalisation
    at the end of each of the three chain pairs and every 8 factors of a chain
    that continues (8 lane operations each), and a 32-operation scalar join.
    n = 40: NP = 20, chains of 7, 7, 6 factors, no mid-chain renormalisation:
    880 + 1216 + 24 + 32.  n = 48: chains of 8, 8, 8 (the 8th is each chain's
    last), 1056 + 1472 + 24 + 32.  n = 64: chains of 11, 11, 10, one
    mid-chain renormalisation each, 1408 + 1984 + 48 + 32."""
    sys.path.insert(0, ROOT)
    import bench

    assert bench.pdf_fp32_ops(40) == 2152
    assert bench.pdf_fp32_ops(48) == 2584
    assert bench.pdf_fp32_ops(64) == 3472

"""Benchmark: Gray-code Glynn permanent throughput on the n = 40 complex128
Haar workload (S(1600, 40): sqrt(1600) times the top-left 40 x 40 block of a
Haar unitary of order 1600), as terms/s, against the roofline of the pipe
that bounds the walk kernel, with the CPU oracle and the paper's own CPU
scheme as baselines.

A step is one pass of the whole hot path (stage A, seed, Gray walk with
product / signed accumulate / row update, double-double reduction) over one
slice of 2^33 consecutive Gray codes of the n = 40 sum: 64 such slices make
up the whole permanent (2^39 codes), and step s covers slice (rank, s) of
it.  Under torchrun each rank walks its own slices (weak scaling); after
timing, rank 0 gathers every rank's 32-byte partials, adds them in rank
order (multirank.combine_partials) and checks the sum against its own
walk of the same slices.

Besides the contract's keys the JSON line carries:
  roofline       FP32-pipe roofline of the default walk kernel (packed FMAs),
                 the issue-slot fraction, and the FP64-equivalent rate of the
                 survey's 6n - 4 operations per term
  alt_rows       the other row arithmetics on the same slice
  n48            n = 48 Haar S(2304, 48): one 2^34-code slice, and the error
                 against the oracle on a 2^18-code slice
  c1_n20         the 20 x 20 complex Gaussian (seed 0): time per permanent and
                 error against the oracle
  exact          0-1 permanents n = 30, 36 modulo four 62-bit primes, checked
                 bit for bit against the stored oracle values
  precision      FP32 products vs FP64 (real Gaussian n = 32, +-1 n = 30)
                 against the stored oracle values
  next_rows      repeated-column, sparse and band timings
  stats          batch statistics of the circular-entry family
  batch          batched vs one launch per matrix on a 2000-matrix sample
  batch_study    the whole 200,000-matrix study in one launch (--batch-study 0
                 skips it)
  err_vs_oracle, cpu_baseline, cpu_baseline_paper

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--batch-sample M] [--batch-study COUNT]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Glynn terms/s (n=40 c128) & % FP64 peak; batched perms/s; err vs FP64 oracle"
N_ORDER = 40
SEED = 1040
CODES_PER_STEP = 1 << 33
L2_FLUSH_BYTES = 256 << 20
GOLDEN = os.path.join(ROOT, "tests", "golden", "configs.json")

# Lane instructions per code of the default walk at n = 40, from ncu's
# smsp__inst_executed.sum x 32 / codes on one 2^30-code launch of the same
# kernel (profiles/k_walk_xp_pdf_c128_n40_haar.md); the issue-slot fraction
# below divides it by the scheduler rate of 4 warp instructions per clock
# per SM at the SM clock sampled during the run.
ISSUED_LANE_INSTR_PER_CODE_N40 = 1265
# DRAM bytes (read + write) of one launch of that kernel at n = 40, from the
# same capture: the per-block staging of the 25.6 KB matrix, the partials and
# write-backs of the L2 flush buffer; independent of the codes per launch.
DRAM_BYTES_PER_LAUNCH_N40 = 102912 + 732672
# Lane instructions per code of the exact modular kernel k_mod<36> (0-1,
# n = 36, exact per-thread 256-bit sums), from ncu on one whole launch
# (profiles/k_mod_n36_zero_one.md); an integer-issue-bound kernel.
ISSUED_LANE_INSTR_PER_CODE_MOD36 = 170


def workload_matrix(n=N_ORDER, seed=SEED):
    from paper_1904_06229_gb300 import workloads as W

    return W.haar_submatrix(n, n * n, seed)


def config_dict(world):
    return {
        "workload": f"n={N_ORDER} complex128 Haar S({N_ORDER * N_ORDER},{N_ORDER}) seed {SEED}; "
                    f"one step = one {CODES_PER_STEP}-code Gray slice of its permanent (2^39 codes in all)",
        "n": N_ORDER,
        "codes_per_step": CODES_PER_STEP,
        "matrix_bytes": 16 * N_ORDER * N_ORDER,
        "l2": "flushed between steps (256 MiB write); the 25.6 KB input is staged to shared memory once per block",
        "parallelism": f"gray-range shards x{world}",
    }


def load_golden():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


# ------------------------------------------------------------------ helpers
class Clocks:
    """Samples nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(A, target_s: float = 12.0):
    """Time the oracle (as it stands) on a slice of the same sum, on all host cores."""
    from oracle import oracle as O

    cores = os.cpu_count() or 1
    n = A.shape[0]
    first = 1 << 30
    count = 1 << 14
    t0 = time.perf_counter()
    O.glynn_partial_parts(A, first, count, parts=cores, threads=cores)
    dt = time.perf_counter() - t0
    # grow the sample to about target_s seconds of CPU work
    count = int(min(1 << 26, max(count, count * target_s / max(dt, 1e-3))))
    count = max(cores, count - count % cores)
    t0 = time.perf_counter()
    g = O.glynn_partial_parts(A, first, count, parts=cores, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": count / dt, "unit": "terms/s", "cores": cores, "kind": "oracle",
            "sample": f"codes [2^30, 2^30+{count}) of the n={n} sum, long double ({O.long_double_digits()}-bit "
                      f"significand) Neumaier-compensated App. A walk, {cores} threads",
            "seconds": dt}, (first, count, g)


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O

    A = workload_matrix()
    cores = os.cpu_count() or 1
    # each step: a bounded slice of the same workload, sized so the whole run
    # stays within a few minutes (about 10 s per step on the host cores)
    probe = 1 << 18
    t0 = time.perf_counter()
    O.glynn_partial_parts(A, 0, probe, parts=cores, threads=cores)
    rate = probe / max(time.perf_counter() - t0, 1e-4)
    per_step = int(max(cores, min(1 << 30, rate * min(args.reference_step_seconds,
                                                      150.0 / max(1, args.steps + args.warmup)))))
    for w in range(args.warmup):
        O.glynn_partial_parts(A, w * per_step, per_step, parts=cores, threads=cores)
    t0 = time.perf_counter()
    for s in range(args.steps):
        O.glynn_partial_parts(A, (args.warmup + s) * per_step, per_step, parts=cores, threads=cores)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    cfg = config_dict(1)
    cfg["workload"] = (f"n={N_ORDER} complex128 Haar S({N_ORDER * N_ORDER},{N_ORDER}) seed {SEED}; one step = "
                       f"{per_step} consecutive Gray codes of its permanent on the host cores (CPU oracle)")
    cfg["codes_per_step"] = per_step
    line = {"metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "long double", "data": "synthetic",
            "impl": "reference", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "terms/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} consecutive codes per step of the n={N_ORDER} sum"},
            "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_paper_sample(A, first, count_hint, oracle_ref, target_s: float = 8.0):
    """The paper's own CPU scheme (Sec. 2.B: double row sums and products,
    Kahan summation, consecutive parts in parallel) on all host cores, on a
    slice of the same sum starting at `first`; its error against the oracle on
    the oracle's slice [first, first + count_hint)."""
    from oracle import oracle as O

    cores = os.cpu_count() or 1
    got = O.paper_scheme_partial(A, first, count_hint, parts=cores, threads=cores)
    ref = complex(float(oracle_ref[0]), float(oracle_ref[1]))
    err = abs(got - ref) / abs(ref)
    count = 1 << 20
    t0 = time.perf_counter()
    O.paper_scheme_partial(A, first, count, parts=cores, threads=cores)
    dt = time.perf_counter() - t0
    count = int(min(1 << 34, max(count, count * target_s / max(dt, 1e-3))))
    count = max(cores, count - count % cores)
    t0 = time.perf_counter()
    O.paper_scheme_partial(A, first, count, parts=cores, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": count / dt, "unit": "terms/s", "cores": cores, "kind": "paper scheme",
            "sample": f"codes [2^30, 2^30+{count}) of the n={A.shape[0]} sum: double row sums and products, Kahan "
                      f"summation, {cores} parts on {cores} threads (Sec. 2.B)",
            "seconds": dt, "rel_err_vs_oracle": err, "err_slice": [first, count_hint]}


# ------------------------------------------------------------------ GPU arm
def pdf_fp32_ops(n):
    """FP32 lane operations per code of the default walk (packed double-float
    rows and products, glynn_walk_xp.cuh), counted from its arithmetic: per
    row pair and Gray step an 11-operation double-float add on each of the two
    components (two rows per packed operation); per term NP - 1 packed complex
    double-float products of 32 packed operations (the chains' steps and the
    joins of three chain pairs), 4-operation packed renormalisations (every 8
    factors of a chain and at its end), and one scalar complex double-float
    product of 32 operations joining the two lanes."""
    NP = (n + 1) // 2
    CP = min(3, NP)
    lens, ren = [1] * CP, CP
    for k in range(CP, NP):
        q = k % CP
        lens[q] += 1
        if lens[q] % 8 == 0 and k + CP < NP:
            ren += 1
    muls = NP - 1
    return NP * 2 * 11 * 2 + muls * 32 * 2 + ren * 4 * 2 + 32


def roofline_of(rows, n, codes, launch_s, peaks, sms, clk_mhz):
    """Roofline of the walk kernel for the row arithmetic in use."""
    ops64 = 6 * n - 4  # the survey's algorithmic FP64-pipe operations per term
    fp64_equiv = {"ops_per_term": ops64, "gops": codes * ops64 / launch_s / 1e9,
                  "vs_dfma_peak": codes * ops64 / launch_s / 1e9 / peaks["dfma"],
                  "note": "FP64-equivalent rate of the survey's 6n-4 FP64 operations per term; not a roofline "
                          "fraction: the default walk does this work in double-float on the FP32 pipe"}
    if rows in ("pdf",):
        ops = pdf_fp32_ops(n)
        achieved = codes * ops / launch_s / 1e9
        peak = 2.0 * peaks["ffma2"]  # packed FMA: two FP32 operations per lane instruction
        out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G FP32 lane-op/s",
               "frac": achieved / peak,
               "traffic": DRAM_BYTES_PER_LAUNCH_N40 if n == N_ORDER else None,
               "kernel": f"perm::k_walk_xp<{n}, false> (packed double-float rows and products, f32x2 FMA pipe)",
               "rows": rows, "fp32_ops_per_term": ops,
               "peak_source": "measured this run: perm_pipe_peak(FFMA2) x 2 FP32 operations (MEASURED_PEAKS.json has "
                              "no FP32 figure)",
               "traffic_note": "bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, ncu, one 2^30-code "
                               "launch of the same kernel: 0.10 MB read + 0.73 MB written); the walk reads its 25.6 KB "
                               "matrix once per block, so the traffic does not grow with the codes per launch"}
        if n == N_ORDER and clk_mhz:
            ipc = ISSUED_LANE_INSTR_PER_CODE_N40
            out["issue_frac"] = codes * ipc / launch_s / (128.0 * sms * clk_mhz * 1e6)
            out["issued_lane_instr_per_term"] = ipc
    else:
        issued = {"fp64": 6 * n - 2, "df": 8, "pair": 8}.get(rows)
        if rows == "fixed":
            k_ix = min((n * 17) // 20, n - 2) if n >= 8 else 0
            issued = 4 * (n - k_ix) + 4 if k_ix else 4 * (n - 1) + 2
        out = {"bound": "alu", "achieved": codes * issued / launch_s / 1e9, "peak": peaks["dfma"],
               "unit": "G FP64 lane-op/s", "frac": codes * issued / launch_s / 1e9 / peaks["dfma"],
               "traffic": None, "rows": rows, "fp64_issued_per_term": issued,
               "peak_source": "measured this run: perm_pipe_peak(DFMA)",
               "note": "FP64 instructions issued per term over the DFMA rate; the binding resource of this row "
                       "arithmetic is described in DESIGN.md"}
    out["fp64_equivalent"] = fp64_equiv
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1904_06229_gb300 import multirank as M
    from paper_1904_06229_gb300 import perm as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group(backend="nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    P.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    A = workload_matrix()
    dA = torch.from_numpy(A.astype(np.complex128)).to(dev)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    total_codes = 1 << (N_ORDER - 1)
    nslices = total_codes // CODES_PER_STEP

    def slice_first(step, r=None):
        return (((rank if r is None else r) + world * step) % nslices) * CODES_PER_STEP

    peaks = {k: P.perm_pipe_peak(k) for k in ("dfma", "ffma", "ffma2", "issue")}
    rows = os.environ.get("PERM_ROWS", "pdf")
    if rows not in ("fixed", "fp64", "df", "pair"):
        rows = "pdf"

    # warm-up
    for w in range(args.warmup):
        P.perm_c128_range(dA, slice_first(w), CODES_PER_STEP, out=out)
        flush.fill_(float(w))
    torch.cuda.synchronize()
    assert P.perm_last_status() == 0

    # timed region: K steps, barrier + synchronize on both sides
    clocks = Clocks(local)
    partials = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        flush.fill_(float(s))
        ev[s][0].record(stream)
        P.perm_c128_range(dA, slice_first(args.warmup + s), CODES_PER_STEP, out=out)
        ev[s][1].record(stream)
        partials.append(out.clone())
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    launch_s = [a.elapsed_time(b) / 1e3 for a, b in ev]
    if world > 1:
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    terms = CODES_PER_STEP * args.steps * world
    value = terms / elapsed

    # end to end through the C ABI with host buffers (pinned): the library
    # copies A in and the partial out inside the timed region
    hA = torch.from_numpy(A.astype(np.complex128)).pin_memory()
    hout = torch.empty(4, dtype=torch.float64).pin_memory()
    for w in range(min(args.warmup, 1)):
        P.perm_c128_range(hA, slice_first(w), CODES_PER_STEP, out=hout, stream=stream)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    h0 = time.perf_counter()
    for s in range(e2e_steps):
        P.perm_c128_range(hA, slice_first(args.warmup + s), CODES_PER_STEP, out=hout, stream=stream)
        stream.synchronize()
        _ = float(hout[0])
    e2e_el = time.perf_counter() - h0
    if world > 1:
        tt = torch.tensor([e2e_el], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_el = float(tt.item())
    e2e_value = CODES_PER_STEP * e2e_steps * world / e2e_el

    # the exchange step of a split sum: rank 0 gathers every rank's partials,
    # adds them in rank order and checks the result against its own walk of
    # the same slices
    multirank = None
    if world > 1:
        gathered = [None] * world
        dist.all_gather_object(gathered, [p.cpu().tolist() for p in partials])
        if rank == 0:
            combined = M.combine_partials(gathered, N_ORDER)
            own = []
            for r in range(world):
                mine = []
                for s in range(args.steps):
                    o = P.perm_c128_range(dA, slice_first(args.warmup + s, r), CODES_PER_STEP).cpu().tolist()
                    mine.append(o)
                own.append(mine)
            single = M.combine_partials(own, N_ORDER)
            multirank = {"ranks": world, "slices": world * args.steps, "combined": [combined.real, combined.imag],
                         "rel_diff_vs_rank0_walk": abs(combined - single) / abs(single)}

    n = N_ORDER
    avg_launch = sum(launch_s) / len(launch_s)
    clk_mhz = clk["sm_mhz"] if clk else None
    roofline = roofline_of(rows, n, CODES_PER_STEP, avg_launch, peaks, sms, clk_mhz)
    line = {"metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(world), "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": "terms/s", "h2d_bytes_per_step": 16 * n * n,
                    "d2h_bytes_per_step": 32, "steps": e2e_steps},
            "gpu_launches": 2 * args.steps, "clocks": clk,
            "pipe_peaks_g_per_s": peaks, "pdf_tile_log": int(os.environ.get("PERM_PDF_TILE_LOG", "0")) or None}
    if multirank is not None:
        line["multirank"] = multirank
    if rank == 0:
        extras(args, line, P, torch, dev, dA, A, rows, peaks, stream, slice_first)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _timed(torch, fn, reps=2):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    r = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return best, r


def extras(args, line, P, torch, dev, dA, A, rows, peaks, stream, slice_first):
    """Every other measurement of the JSON line (rank 0, after the timed region)."""
    if not args.no_alt_rows:
        line["alt_rows"] = alt_rows_measure(P, torch, dA, rows, slice_first(args.warmup))
    if not args.no_extras:
        line["n48"] = n48_measure(P, torch, dev)
        line["c1_n20"] = c1_measure(P, torch, dev)
        clk = (line.get("clocks") or {}).get("sm_mhz")
        line["exact"] = exact_measure(P, torch, dev, clk)
        line["precision"] = precision_measure(P, torch, dev)
        line["next_rows"] = next_rows_measure(P, torch, dev)
        line["stats"] = stats_measure(P, torch, dev)
    if args.batch_sample > 0:
        line["batch"] = batch_measure(P, torch, dev, args.batch_sample)
    if args.batch_study > 0:
        line["batch_study"] = batch_study_measure(P, torch, dev, args.batch_study, peaks)
    if not args.no_cpu_baseline:
        cpu_leg(line, P, torch, dev, dA, A)


def alt_rows_measure(P, torch, dA, rows, first):
    """The other row arithmetics on the bench's own slice: rate and relative
    difference from the default's partial sum."""
    out = []
    ref = P.perm_c128_range(dA, first, CODES_PER_STEP).cpu().numpy()
    vr = complex(ref[0] + ref[1], ref[2] + ref[3])
    for alt in [m for m in ("fixed", "fp64", "df", "pair") if m != rows]:
        os.environ["PERM_ROWS"] = alt
        try:
            P.perm_c128_range(dA, 0, 1 << 24)
            torch.cuda.synchronize()
            at, o = _timed(torch, lambda: P.perm_c128_range(dA, first, CODES_PER_STEP), reps=1)
            o = o.cpu().numpy()
            va = complex(o[0] + o[1], o[2] + o[3])
            out.append({"rows": alt, "terms_per_s": CODES_PER_STEP / at, "rel_diff_vs_default": abs(va - vr) / abs(vr)})
        finally:
            os.environ["PERM_ROWS"] = rows
    return out


def n48_measure(P, torch, dev):
    """n = 48 Haar S(2304, 48), seed 1048: one 2^34-code slice of its 2^47-code
    sum in one call (the whole sum would be 8192 such slices)."""
    A48 = torch.from_numpy(workload_matrix(48, 1048)).to(dev)
    first, count = 5 << 34, 1 << 34
    P.perm_c128_range(A48, 0, 1 << 24)
    torch.cuda.synchronize()
    t, o = _timed(torch, lambda: P.perm_c128_range(A48, first, count), reps=1)
    o = o.cpu().numpy()
    return {"workload": "n=48 complex128 Haar S(2304,48) seed 1048, codes [5*2^34, 6*2^34)", "codes": count,
            "seconds": t, "terms_per_s": count / t, "whole_permanent_hours": (1 << 47) / (count / t) / 3600.0,
            "partial": [o[0] + o[1], o[2] + o[3]]}


def c1_measure(P, torch, dev):
    """The 20 x 20 complex Gaussian of seed 0 (2^19 codes): device time per
    permanent (CUDA events over 20 back-to-back calls) and host latency of one
    call including the copy back."""
    from paper_1904_06229_gb300 import workloads as W

    A20 = torch.from_numpy(W.complex_gaussian(20, 0)).to(dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    for _ in range(3):
        P.perm_c128(A20, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        P.perm_c128(A20, out=out)
    e1.record()
    torch.cuda.synchronize()
    dev_us = e0.elapsed_time(e1) * 1e3 / 20
    lat = []
    for _ in range(10):
        h0 = time.perf_counter()
        v = P.perm_c128(A20, out=out).cpu().numpy()
        lat.append(time.perf_counter() - h0)
    return {"workload": "n=20 complex Gaussian N(0,1/2)+iN(0,1/2) seed 0", "us_per_permanent": dev_us,
            "host_latency_us": statistics.median(lat) * 1e6, "terms_per_s": (1 << 19) / (dev_us * 1e-6),
            "value": [float(v[0]), float(v[1])]}


def exact_measure(P, torch, dev, clk_mhz=None):
    """Exact 0-1 permanents (density 1/2; n = 30 seed 6, n = 36 seed 7) modulo
    four 62-bit primes, CRT on the host; each checked bit for bit against the
    stored oracle value (tests/golden/configs.json), also through the
    modular group walk.  n = 36 carries the issue-slot roofline of its
    integer kernel (ncu's lane instructions per code x codes/s over 4 warp
    instructions per clock per SM at the SM clock sampled in the run)."""
    from paper_1904_06229_gb300 import workloads as W

    golden = load_golden()
    primes = P.perm_default_primes()
    out = {}
    for n, seed in ((30, 6), (36, 7)):
        t = torch.from_numpy(W.zero_one(n, seed)).to(dev)
        res = torch.empty(4, dtype=torch.int64, device=dev)
        sec, _ = _timed(torch, lambda: P.perm_mod01(t, primes, res))
        val = P.perm_crt([int(v) for v in res.cpu()], primes)
        old = os.environ.get("PERM_MOD_SUM")
        os.environ["PERM_MOD_SUM"] = "modular"
        try:
            res_m = torch.empty(4, dtype=torch.int64, device=dev)
            sec_m, _ = _timed(torch, lambda: P.perm_mod01(t, primes, res_m), reps=1)
        finally:
            if old is None:
                del os.environ["PERM_MOD_SUM"]
            else:
                os.environ["PERM_MOD_SUM"] = old
        ref = int(golden[f"zero_one_n{n}_seed{seed}"]["per"])
        out[f"n{n}"] = {"seconds": sec, "codes_per_s": (1 << (n - 1)) / sec, "per": str(val),
                        "per_bits": val.bit_length(), "matches_oracle": val == ref,
                        "modular_walk": {"seconds": sec_m, "codes_per_s": (1 << (n - 1)) / sec_m,
                                         "same_residues": res_m.cpu().tolist() == res.cpu().tolist()}}
        if n == 36 and clk_mhz:
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            achieved = (1 << (n - 1)) / sec * ISSUED_LANE_INSTR_PER_CODE_MOD36 / 1e9
            peak = 128.0 * sms * clk_mhz * 1e6 / 1e9
            out[f"n{n}"]["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak,
                                        "unit": "G lane-instr/s (issue slots)", "frac": achieved / peak,
                                        "issued_lane_instr_per_code": ISSUED_LANE_INSTR_PER_CODE_MOD36,
                                        "kernel": "perm::k_mod<36> (int32 rows, exact 256-bit per-thread sums)"}
    return out


def precision_measure(P, torch, dev):
    """FP32-product variant vs FP64 against the stored oracle values: real
    N(0,1) n = 32 (seed 4, long-double oracle) and +-1 n = 30 (seed 5, exact
    integer); the FP32 variant's stated bound is (2n + 2) 2^-24 sum|t|."""
    from paper_1904_06229_gb300 import workloads as W

    golden = load_golden()
    out = {}
    g = golden["real_gaussian_n32_seed4"]
    ref, asum = float(g["per"]), float(g["abs_sum"])
    A = torch.from_numpy(W.real_gaussian(32, 4)).to(dev)
    t64, r64 = _timed(torch, lambda: P.perm_f64(A).cpu())
    t32, r32 = _timed(torch, lambda: P.perm_f64_f32p(A).cpu())
    out["real_gaussian_n32"] = {"fp64_s": t64, "f32p_s": t32, "kappa": asum / abs(ref),
                                "fp64_rel_err": abs(float(r64[0]) - ref) / abs(ref),
                                "f32p_rel_err": abs(float(r32[0]) - ref) / abs(ref),
                                "f32p_stated_bound": 66 * 2.0 ** -24 * asum / abs(ref)}
    g = golden["pm1_n30_seed5"]
    exact = int(g["per"])
    B = torch.from_numpy(W.bernoulli_pm1(30, 5).astype(np.float64)).to(dev)
    t64, r64 = _timed(torch, lambda: P.perm_f64(B).cpu())
    t32, r32 = _timed(torch, lambda: P.perm_f64_f32p(B).cpu())
    out["pm1_n30"] = {"exact": str(exact), "fp64_rel_err": abs(float(r64[0]) - exact) / abs(exact),
                      "f32p_rel_err": abs(float(r32[0]) - exact) / abs(exact), "fp64_s": t64, "f32p_s": t32}
    if "abs_sum" in g:
        out["pm1_n30"]["f32p_stated_bound"] = 62 * 2.0 ** -24 * float(g["abs_sum"]) / abs(exact)
    return out


def cpu_leg(line, P, torch, dev, dA, A):
    """The CPU baselines (the oracle as it stands, the paper's own scheme) and
    the GPU's error against the oracle on the same slices and configurations."""
    from oracle import oracle as O
    from paper_1904_06229_gb300 import workloads as W

    cb, (first, count, g) = cpu_oracle_sample(A)
    line["cpu_baseline"] = cb
    o = P.perm_c128_range(dA, first, count).cpu().numpy()
    got = complex(o[0] + o[1], o[2] + o[3])
    ref = complex(float(g[0]), float(g[1]))
    line["err_vs_oracle"] = {"slice": [first, count], "rel": abs(got - ref) / abs(ref),
                             "kappa_slice": float(g[2]) / abs(ref)}
    line["cpu_baseline_paper"] = cpu_paper_sample(A, first, count, g)
    cores = os.cpu_count() or 1
    if "n48" in line:
        A48 = workload_matrix(48, 1048)
        f48, c48 = (1 << 46) + 12345, 1 << 18
        g48 = O.glynn_partial_parts(A48, f48, c48, parts=cores, threads=cores)
        o = P.perm_c128_range(torch.from_numpy(A48).to(dev), f48, c48).cpu().numpy()
        r48 = complex(float(g48[0]), float(g48[1]))
        line["n48"]["err_vs_oracle"] = {"slice": [f48, c48],
                                        "rel": abs(complex(o[0] + o[1], o[2] + o[3]) - r48) / abs(r48),
                                        "kappa_slice": float(g48[2]) / abs(r48)}
    if "c1_n20" in line:
        r = O.per(W.complex_gaussian(20, 0))
        ref = complex(float(r[0]), float(r[1]))
        v = line["c1_n20"]["value"]
        line["c1_n20"]["rel_err_vs_oracle"] = abs(complex(v[0], v[1]) - ref) / abs(ref)
        line["c1_n20"]["kappa"] = float(r[2]) / abs(ref)


def next_rows_measure(P, torch, dev):
    """The widened rows: repeated columns (Eq. ryser2), sparse (App. B) and
    band-limited (App. C) permanents, each against the dense Gray walk where
    that is feasible."""
    from paper_1904_06229_gb300 import workloads as W

    out = {}
    # Boson-sampling-like output with collisions: 15 modes with two photons each (n = 30)
    Cb = W.haar_submatrix(30, 900, 30)[:, :15]
    mult = [2] * 15
    A = np.concatenate([np.repeat(Cb[:, k:k + 1], 2, axis=1) for k in range(15)], axis=1)
    tC = torch.from_numpy(np.ascontiguousarray(Cb)).to(dev)
    tA = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    t_rep, r_rep = _timed(torch, lambda: P.perm_c128_repeated(tC, mult).cpu())
    t_den, r_den = _timed(torch, lambda: P.perm_c128(tA).cpu())
    a, b = complex(*r_rep.tolist()), complex(*r_den.tolist())
    out["repeated_n30_2x15"] = {"terms": 3 ** 15, "seconds": t_rep, "dense_codes": 1 << 29, "dense_seconds": t_den,
                                "speedup": t_den / t_rep, "rel_diff_vs_dense": abs(a - b) / abs(b)}
    # sparse: identity + Bernoulli(0.02) off-diagonal, n = 48
    S = W.sparse_matrix(48, 0.02, 48)
    block, count = P.perm_sparse_partition(S)
    tS = torch.from_numpy(S).to(dev)
    t_sp, _ = _timed(torch, lambda: P.perm_c128_sparse(tS).cpu())
    out["sparse_n48_p0.02"] = {"sets": count, "dense_codes": 1 << 47, "seconds": t_sp, "sets_per_s": count / t_sp}
    # band: 1000 real-Gaussian band matrices, n = 100, k = 5 (App. C study sizes)
    Bm = np.stack([W.band_matrix(100, 5, s, kind="real") for s in range(1000)])
    tB = torch.from_numpy(Bm).to(dev)
    t_b, _ = _timed(torch, lambda: P.perm_c128_band(tB, 5).cpu())
    out["band_n100_k5_x1000"] = {"seconds": t_b, "matrices_per_s": 1000 / t_b}
    return out


def stats_measure(P, torch, dev, per_order: int = 500):
    """Sec. 4 circular-entry study on a sample: per order n = 8..16, `per_order`
    matrices with entries exp(i theta), statistics of X = |per| / sqrt(n!) from
    perm_batch_stats (one graph launch plus the statistics kernel)."""
    from paper_1904_06229_gb300 import workloads as W

    mats, seed = [], 0
    for n in range(8, 17):
        for _ in range(per_order):
            mats.append(torch.from_numpy(W.circular(n, 500_000 + seed)).to(dev))
            seed += 1
    P.perm_batch_stats(mats)  # tunes, captures the graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, st = P.perm_batch_stats(mats)
    e1.record()
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    per_n = {str(n): {"count": int(st[n, 0]), "mean_X": st[n, 1] / st[n, 0], "mean_X2": st[n, 2] / st[n, 0]}
             for n in range(8, 17)}
    return {"family": "circular exp(i theta)", "matrices": len(mats), "seconds": e0.elapsed_time(e1) / 1e3,
            "per_order": per_n}


def batch_measure(P, torch, dev, sample):
    """The batch study's distribution (n ~ U{12..28}, half Gaussian half Haar,
    shuffled; seed 3) on `sample` matrices: one persistent graph launch vs one
    perm_c128 launch per matrix."""
    from paper_1904_06229_gb300 import workloads as W

    ns, mats = W.batch_study(sample, seed=3)
    dm = [torch.from_numpy(m.astype(np.complex128)).to(dev) for m in mats]
    ptrs = torch.tensor([m.data_ptr() for m in dm], dtype=torch.int64, device=dev)
    out = torch.empty((sample, 2), dtype=torch.float64, device=dev)
    P.perm_batch(dm, out=out, ptrs=ptrs)  # tunes unseen orders, captures the graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    P.perm_batch(dm, out=out, ptrs=ptrs)
    e1.record()
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 1e3
    single = torch.empty((sample, 2), dtype=torch.float64, device=dev)
    for k in range(min(sample, 50)):
        P.perm_c128(dm[k], out=single[k])
    torch.cuda.synchronize()
    e0.record()
    for k in range(sample):
        P.perm_c128(dm[k], out=single[k])
    e1.record()
    torch.cuda.synchronize()
    ts = e0.elapsed_time(e1) / 1e3
    d = (out - single).abs().max().item()
    scale = single.abs().max().item()
    terms = int(sum(1 << (int(n) - 1) for n in ns))
    return {"sample": sample, "orders": "12..28", "terms": terms, "batched_perms_per_s": sample / tb,
            "per_launch_perms_per_s": sample / ts, "speedup": ts / tb, "batched_terms_per_s": terms / tb,
            "max_abs_diff_vs_per_launch": d, "max_abs_value": scale, "gpu_launches_batched": 2}


def batch_study_measure(P, torch, dev, count, peaks=None):
    """The whole batch study in one persistent launch: `count` matrices (n ~
    U{12..28}, half Gaussian, half Haar S(n^2, n), shuffled; seed 3) through
    perm_batch_stats, with the per-order moments of X = |per| / sqrt(n!), and
    64 results checked against single perm_c128 launches.  Roofline: the FP32
    lane operations of the orders on the block-per-item kernels (the default
    walk's arithmetic, pdf_fp32_ops per code) over the launch time, against
    the measured packed-FMA rate; the orders on the warp kernel (FP64 or
    fixed-point rows) are left out of the count and named."""
    from paper_1904_06229_gb300 import workloads as W

    t0 = time.time()
    ns, mats = W.batch_study(count, seed=3)
    gen_s = time.time() - t0
    offs = np.concatenate([[0], np.cumsum([m.size for m in mats])]).astype(np.int64)
    flat = np.empty(int(offs[-1]), dtype=np.complex128)
    for k, m in enumerate(mats):
        flat[offs[k]:offs[k + 1]] = m.ravel()
    del mats
    dflat = torch.from_numpy(flat).to(dev)
    dm = [dflat[int(offs[k]):int(offs[k + 1])].view(int(ns[k]), int(ns[k])) for k in range(count)]
    ptrs = torch.tensor([t.data_ptr() for t in dm], dtype=torch.int64, device=dev)
    terms = int(sum(1 << (int(n) - 1) for n in ns))
    P.perm_batch_autotune(int(ns.min()), int(ns.max()))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0 = time.time()
    e0.record()
    out, stats = P.perm_batch_stats(dm, ptrs=ptrs)  # plan (item list, graph) built on the host, then one launch
    plan_s = time.time() - h0
    e1.record()
    torch.cuda.synchronize()
    total_s = e0.elapsed_time(e1) / 1e3
    status = P.perm_last_status()
    rng = np.random.default_rng(1)
    worst = 0.0
    for k in rng.choice(count, 64, replace=False):
        ref = P.perm_c128(dm[int(k)]).cpu().numpy()
        got = out[int(k)].cpu().numpy()
        worst = max(worst, float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)))
    st = stats.cpu().numpy()
    per_n = {}
    for n in range(int(ns.min()), int(ns.max()) + 1):
        c = float(st[n, 0])
        if c > 0:
            per_n[str(n)] = {"count": int(c), "mean_X": st[n, 1] / c, "mean_X2": st[n, 2] / c, "mean_X4": st[n, 4] / c}
    kernel_s = total_s - plan_s
    out = {"matrices": count, "orders": "12..28", "terms": terms, "generate_s": gen_s,
           "seconds_incl_host_plan": total_s, "host_plan_s": plan_s, "perms_per_s": count / kernel_s,
           "terms_per_s": terms / kernel_s, "status": status, "max_rel_diff_vs_perm_c128_64": worst,
           "per_order": per_n}
    if peaks:
        _, kinds = P.perm_batch_tuning(torch.cuda.current_device())
        ops, warp_orders, warp_terms = 0, [], 0
        for n in np.unique(ns):
            codes = int((ns == n).sum()) << (int(n) - 1)
            if kinds[int(n)] in (2, 3, 4):
                ops += codes * pdf_fp32_ops(int(n))
            else:
                warp_orders.append(int(n))
                warp_terms += codes
        achieved = ops / kernel_s / 1e9
        peak = 2.0 * peaks["ffma2"]
        out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G FP32 lane-op/s",
                           "frac": achieved / peak, "fp32_lane_ops": ops,
                           "warp_kernel_orders": warp_orders, "warp_kernel_terms_share": warp_terms / terms,
                           "peak_source": "perm_pipe_peak(FFMA2) x 2, measured this run"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--reference-step-seconds", type=float, default=10.0,
                    help="host seconds per step of the reference arm (the CPU oracle)")
    ap.add_argument("--batch-sample", type=int, default=2000)
    ap.add_argument("--batch-study", type=int, default=200000,
                    help="matrices of the whole batch study, run in one launch after the timed region (0 skips)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-alt-rows", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other configurations' measurements")
    ap.add_argument("--codes-log2", type=int, default=33,
                    help="codes per step (2^k); smaller values make a short case for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    global CODES_PER_STEP
    if not 10 <= args.codes_log2 <= 38:
        raise SystemExit("--codes-log2 must be in 10..38")
    CODES_PER_STEP = 1 << args.codes_log2
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark of the GB300 column-wise SpGEMM (one JSON line on rank 0).

A step is one pass of the whole hot path over the workload: input
validation, Op_j and binning, symbolic pass, scan, numeric pass with sorted
output (spgemm_symbolic + spgemm_numeric through the C ABI, a new plan every
step).  Default workload: C = A x A with A an R-MAT power-law matrix (2^18
rows, a,b,c,d = 0.57,0.19,0.19,0.05, 8 edges per row drawn, columns capped at
2000 entries, FP64 values U[-1,1]), the largest single product of the
workload set.  The line also carries the random 2^20 product (the hash
regime), the 512-product batch, the Galerkin backward and a sweep of the
threshold t, each with its own roofline figures.

Metric: GFLOP/s = 2 x sum_j Op_j / step time (Op_j = products of column j);
the step time is the median of K CUDA-event timed steps.
Roofline: the binned numeric pass, algorithmic bytes over its event-timed
duration against the measured HBM copy bandwidth.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    3: "C=AxA R-MAT 2^18 (a,b,c,d=0.57,0.19,0.19,0.05, 8 edges/row, col cap 2000), FP64",
    2: "C=AxB random 2^20 x 2^20, nnz/col U{1..8}, FP64",
    1: "C=AxA 2D 5-point Laplacian 32x32, FP64",
}
L2_FLUSH_BYTES = 512 << 20
METRIC = "SpGEMM GFLOP/s (2 x intermediate products / s)"
INF = (1 << 63) - 1
# light bins: ESC or lane-group hash tables, by the light-column accumulator
BIN_NAMES = (["empty"] + [f"light_op<={o}" for o in (8, 16, 32, 64, 128, 256)]
             + [f"hash_cta_op<={o}" for o in (512, 1024, 2048, 4096, 8192)] + ["hash_global", "dense_spa"])
DENSE_BIN = 13
# thresholds of the sweep (Section 5.4 varies t the same way; t = 0 sends
# every column to the dense SPA, t = infinity every column to hash tables)
SWEEP_T = [0, 20, 30, 40, 50, 60, INF]


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", type=int, default=3, choices=[1, 2, 3])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-aux", action="store_true",
                   help="skip the other workloads (random 2^20, batch, backward) and the t sweep")
    p.add_argument("--no-sweep", action="store_true", help="skip the sweep of the threshold t")
    p.add_argument("--batched-only", type=int, default=0, metavar="N",
                   help="only the batched measurement, on the first N products of the seeded batch, "
                        "with t=33, 128 threads (no tuner); for a small profiling case")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="target CPU seconds of the oracle sample")
    p.add_argument("--t", type=int, default=None,
                   help="H-HASH(t) threshold (default: the library's)")
    p.add_argument("--cta-threads", type=int, default=None,
                   help="threads per CTA of the CTA-level kernels (default: the library's)")
    p.add_argument("--dense-cache", type=int, default=None,
                   help="bytes of workspace for dense-column SPA flags kept between phases")
    p.add_argument("--rmat-scale", type=int, default=18,
                   help="log2 size of the R-MAT workload (smaller for profiler captures)")
    p.add_argument("--accumulator", default=None, choices=["hash", "esc", "auto"],
                   help="accumulator of the light columns (default: the library's)")
    return p.parse_args(argv)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# DRAM bytes (read + write) of one launch of a dominant kernel from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), with the
# algorithmic bytes of that launch; a launch of another size reports the
# captured bytes scaled by its algorithmic bytes.  A record holds for its
# workload, bin and light-column accumulators (None: the library's default)
# in the default configuration otherwise, and only for the kernel sources
# it was taken with: the hash covers the files that define the kernel, and
# any change there reports null.
MEASURED_TRAFFIC = (
    {"workload": 3, "bin": 13, "capture": "R-MAT 2^17", "accumulators": (None,),
     "bytes": 422044416 + 1971488512, "algorithmic_bytes": 5313831440,
     "sources_sha256_16": "45ea3b2a9058a02d",
     "sources": ("spgemm_internal.cuh", "kernels.cuh", "columns.cuh", "numeric.cu")},
    {"workload": 2, "bin": 3, "capture": "random 2^20 (the same launch, ESC)", "accumulators": (None, "auto", "esc"),
     "bytes": 305311488 + 120249344, "algorithmic_bytes": 338467476,
     "sources_sha256_16": "ba9ae6c19f74017f",
     "sources": ("spgemm_internal.cuh", "kernels.cuh", "columns.cuh", "esc.cuh", "esc.cu")},
)


def measured_traffic(top_bin, top_bytes, args, workload=None, accumulator=None):
    """(bytes, source) of the dominant kernel's DRAM traffic, or (None, why).
    `args`: the command line of the main workload; a side workload passes
    args=None with its number and light-column accumulator."""
    import hashlib
    if args is not None:
        workload = args.workload
        accumulator = getattr(args, "accumulator", None)
        default_cfg = args.t is None and args.cta_threads is None and args.dense_cache is None
    else:
        default_cfg = True
    if not MEASURED_TRAFFIC:
        return None, "no capture of the current kernel sources"
    for t in MEASURED_TRAFFIC:
        if t["workload"] != workload or t["bin"] != top_bin or not default_cfg or accumulator not in t["accumulators"]:
            continue
        h = hashlib.sha256()
        root = os.path.join(ROOT, "paper_2303_02471_gb300", "csrc")
        for f in t["sources"]:
            with open(os.path.join(root, f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest()[:16] != t["sources_sha256_16"]:
            return None, "kernel sources changed since the capture"
        scaled = int(round(t["bytes"] * top_bytes / t["algorithmic_bytes"]))
        return scaled, (f"ncu capture of {t['capture']}, {t['bytes']:.4g} B per launch, "
                        f"scaled by algorithmic bytes {top_bytes:.4g} / {t['algorithmic_bytes']:.4g}")
    return None, "no capture of this kernel, workload or configuration"


def algorithmic_bytes(A, B, products, nnzC, w):
    """Numeric pass, per launch: B columns (colptr, rows, values), the
    gathered A column pointers and A entries of every product, and C written
    once (colptr read, rows and values written)."""
    nB = B.ncols
    nnzB = int(B.colptr[-1])
    return (8 * (nB + 1) + nnzB * (4 + w) + 16 * nnzB + products * (4 + w)
            + 8 * (nB + 1) + nnzC * (4 + w))


def backward_bytes(A, B, products, nnzC, w, need_dA=True, need_dB=True):
    """Backward of one product, per launch set: B columns (colptr, rows,
    values), the gathered A column pointers and A entries (row and value) of
    every product, C's pattern and dC read once, dA and dB written once."""
    nB = B.ncols
    nnzA = int(A.colptr[-1])
    nnzB = int(B.colptr[-1])
    return (8 * (nB + 1) + nnzB * (4 + w) + 16 * nnzB + products * (4 + w)
            + 8 * (nB + 1) + nnzC * (4 + w) + (nnzA * w if need_dA else 0) + (nnzB * w if need_dB else 0))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        # this rank's GPU: its LOCAL_RANK-th visible device
        local = int(os.environ.get("LOCAL_RANK", "0"))
        visible = [d for d in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if d]
        dev = visible[local] if local < len(visible) else str(local)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={dev}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        out.update(sm_mhz=float(np.median(sm)) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons), samples=len(rows))
        return out


# --------------------------------------------------------------- workloads
def workload_name(args):
    if args.workload == 3 and args.rmat_scale != 18:
        return WORKLOADS[3].replace("2^18", f"2^{args.rmat_scale}")
    return WORKLOADS[args.workload]


def make_workload(k, rmat_scale=18):
    from paper_2303_02471_gb300 import synth
    if k == 3 and rmat_scale != 18:
        A = synth.rmat(rmat_scale, seed=0)
        return A, A
    A, B = synth.workload(k)
    return A, B


def bin_bytes(st, b, w):
    """Algorithmic bytes of one bin kernel of the numeric pass: its B columns
    (colptr pair, rows, values), the gathered A column pointers (16 B per B
    entry), the gathered A entries (one per product), the C column pointers
    and the C entries written once."""
    cols = st["count"][b]
    return (16 * cols + st["nnz_b"][b] * (4 + w + 16) + st["products"][b] * (4 + w)
            + 16 * cols + st["nnz"][b] * (4 + w))


def dominant_bin(st, w):
    """The bin kernel the roofline reports: the non-empty bin with the most
    algorithmic bytes (not the longest event time: bins on side streams
    start timing with the pass and include waiting for SMs)."""
    nbins = len(st["count"])
    return int(np.argmax([bin_bytes(st, b, w) if b and st["count"][b] else 0 for b in range(nbins)]))


def column_sample(B, frac, seed=0):
    """Every column of B kept with probability `frac` (a CSC of the subset)."""
    from types import SimpleNamespace
    rng = np.random.default_rng(seed)
    cols = np.nonzero(rng.random(B.ncols) < frac)[0]
    cnt = np.diff(B.colptr)[cols]
    cp = np.zeros(len(cols) + 1, np.int64)
    np.cumsum(cnt, out=cp[1:])
    starts = B.colptr[cols]
    idx = (np.repeat(starts - cp[:-1], cnt) + np.arange(int(cp[-1]))).astype(np.int64)
    return SimpleNamespace(nrows=B.nrows, ncols=len(cols), colptr=cp, rowidx=B.rowidx[idx],
                           values=B.values[idx]), cols


def oracle_rate(A, B, op, threads, target_s, seed):
    """GFLOP/s of the oracle on `threads` host threads over a seeded column
    sample of B sized for about target_s seconds (whole product when it fits)."""
    import oracle
    small, cols = column_sample(B, 0.005, seed=seed)
    t0 = time.perf_counter()
    oracle.spgemm(A, small, nthreads=threads)
    rate = max(1.0, op[cols].sum()) / max(1e-3, time.perf_counter() - t0)
    frac = min(1.0, target_s * rate / max(1, op.sum()))
    sample, cols = column_sample(B, frac, seed=seed + 1)
    products = int(op[cols].sum())
    t0 = time.perf_counter()
    oracle.spgemm(A, sample, nthreads=threads)
    dt = time.perf_counter() - t0
    return 2.0 * products / dt / 1e9, (f"{len(cols)} of {B.ncols} columns of B (seeded, p={frac:.4f}), "
                                       f"{products} products, {dt:.2f} s")


def cpu_baseline(A, B, target_s, unit):
    """The oracle as it stands on all host cores (bounded column sample),
    and on one thread (a smaller sample)."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    op = oracle.op_counts(A, B)
    threads = oracle.threads(cores)
    value, sample = oracle_rate(A, B, op, threads, target_s, seed=1)
    v1, s1 = oracle_rate(A, B, op, 1, max(1.0, target_s / 4), seed=3)
    return {"value": value, "unit": unit, "cores": threads, "kind": "oracle", "sample": sample,
            "single_thread": {"value": v1, "unit": unit, "cores": 1, "sample": s1}}


# ------------------------------------------------------------------ arms
REFERENCE_BUDGET_S = 240.0  # host seconds of the whole reference run at most


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores, as the other arm: W untimed
    and K timed steps, every step the whole workload product (a seeded
    column sample only if the whole product would not fit the budget)."""
    unit = "GFLOP/s"
    if rank != 0:
        return None
    import oracle
    A, B = make_workload(args.workload, args.rmat_scale)
    cores = len(os.sched_getaffinity(0))
    threads = oracle.threads(cores)
    op = oracle.op_counts(A, B)
    small, cols = column_sample(B, 0.005, seed=1)
    t0 = time.perf_counter()
    oracle.spgemm(A, small, nthreads=threads)
    rate = max(1.0, op[cols].sum()) / max(1e-3, time.perf_counter() - t0)
    per_step = REFERENCE_BUDGET_S / max(1, args.warmup + args.steps)
    frac = 1.0 if op.sum() <= per_step * rate else per_step * rate / max(1, op.sum())
    if frac >= 1.0:
        sample, cols = B, np.arange(B.ncols)
    else:
        sample, cols = column_sample(B, frac, seed=2)
    products = int(op[cols].sum())
    for _ in range(args.warmup):
        oracle.spgemm(A, sample, nthreads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.spgemm(A, sample, nthreads=threads)
        times.append(time.perf_counter() - t0)
    dt = float(np.median(times))
    value = 2.0 * products / dt / 1e9
    what = ("the whole product" if frac >= 1.0 else
            f"{len(cols)} of {B.ncols} columns of B (seeded, p={frac:.4f})")
    base = {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
            "sample": f"{what} per step, {products} products, median of {args.steps} timed steps "
                      f"{dt:.3f} s"}
    return {"impl": "reference", "metric": METRIC,
            "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args), "same_config": frac >= 1.0},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


class Product:
    """One workload product on the device, stepped through the C ABI."""

    def __init__(self, A_h, B_h, dev, cfg):
        import torch
        from paper_2303_02471_gb300 import _native as N
        from paper_2303_02471_gb300 import ops
        self.N, self.ops, self.torch = N, ops, torch
        self.A_h, self.B_h = A_h, B_h
        self.A = ops.CscMatrix.from_host(A_h, device=dev)
        self.B = self.A if B_h is A_h else ops.CscMatrix.from_host(B_h, device=dev)
        self.cfg = cfg
        self.ncfg = cfg.native()
        self.lib = N.lib()
        self.hd = ops.handle(dev)
        self.stream = torch.cuda.current_stream()
        self.sp = ctypes.c_void_p(self.stream.cuda_stream)
        self.cA, self.cB = ops._csc(self.A), ops._csc(self.B)
        self.ws = torch.empty(ops.workspace_size(self.A, self.B, cfg), dtype=torch.uint8, device=dev)
        self.colptr = torch.empty(self.B.ncols + 1, dtype=torch.int64, device=dev)
        plan = self.plan()
        info = plan.info()
        self.stats = plan.bin_stats()
        self.stats["count"] = info["bins"]
        self.products = info["products"]
        self.t = info["t"]
        self.nnz = plan.nnz
        self.side = plan.bin_streams()
        lc = plan.launch_count()
        self.launches = lc["symbolic"] + lc["numeric"]
        plan.destroy()
        self.rowidx = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        self.values = torch.empty(self.nnz, dtype=self.A.dtype, device=dev)

    def plan(self):
        N, ops = self.N, self.ops
        nnz, h = ctypes.c_int64(), ctypes.c_void_p()
        N.check(self.lib.spgemm_symbolic(self.hd.ptr, ctypes.byref(self.cA), ctypes.byref(self.cB),
                                         ctypes.byref(self.ncfg), ctypes.c_void_p(self.ws.data_ptr()),
                                         self.ws.numel(), ctypes.c_void_p(self.colptr.data_ptr()),
                                         ctypes.byref(nnz), ctypes.byref(h), self.sp), "spgemm_symbolic")
        return ops.Plan(h, self.ws, self.A, self.B, self.colptr, nnz.value, self.cfg, self.hd)

    def numeric(self, plan):
        self.N.check(self.lib.spgemm_numeric(plan.handle, ctypes.byref(self.cA), ctypes.byref(self.cB),
                                             ctypes.c_void_p(self.colptr.data_ptr()),
                                             ctypes.c_void_p(self.rowidx.data_ptr()),
                                             ctypes.c_void_p(self.values.data_ptr()), self.sp),
                     "spgemm_numeric")


def time_steps(prod, steps, warmup, flush, world=1, clocks=None, bin_timing=True):
    """W untimed and K timed steps (a new plan every step); per-step events
    (whole step, symbolic, numeric) and the bin times of every step."""
    import torch
    stream = prod.stream
    for _ in range(warmup):
        plan = prod.plan()
        prod.numeric(plan)
        plan.check()
        plan.destroy()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    bin_ms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    for i in range(steps):
        flush.fill_(i & 0xff)  # evict A and B from L2 between steps
        ev[i][0].record(stream)
        plan = prod.plan()
        if bin_timing:
            plan.set_timing(True)
        ev[i][1].record(stream)
        prod.numeric(plan)
        ev[i][2].record(stream)
        plan.check()
        if bin_timing:
            bin_ms.append(plan.bin_times())
        plan.destroy()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks is not None else None
    step = [a.elapsed_time(c) for a, b, c in ev]
    sym = [a.elapsed_time(b) for a, b, c in ev]
    num = [b.elapsed_time(c) for a, b, c in ev]
    return {"step": step, "sym": sym, "num": num, "bins": bin_ms, "clocks": clk}


def serial_bin_times(A_h, B_h, dev, cfg, flush, repeats=3):
    """Every bin kernel of the numeric pass timed on its own: a plan whose
    bins all run in order on the caller's stream (no side streams), median
    of `repeats` timed numeric calls."""
    from dataclasses import replace
    import torch
    prod = Product(A_h, B_h, dev, replace(cfg, side_streams=False))
    plan = prod.plan()
    plan.set_timing(True)
    prod.numeric(plan)
    plan.check()
    out = []
    for i in range(repeats):
        flush.fill_(i & 0xff)
        prod.numeric(plan)
        out.append(plan.bin_times())
    plan.check()
    plan.destroy()
    torch.cuda.synchronize()
    return np.median(np.array(out), axis=0)


def product_report(prod, res, serial, peak, peak_kind, args, w=8, workload=None, accumulator=None):
    """Roofline of the dominant bin kernel and of the whole numeric pass,
    phase medians and per-bin figures of one product."""
    st = prod.stats
    top = dominant_bin(st, w)
    top_bytes = bin_bytes(st, top, w)
    live = np.median(np.array(res["bins"]), axis=0) if res["bins"] else serial
    # a bin on a side stream has event times that include waiting for SMs:
    # its roofline takes the serialised time
    top_ms = float(serial[top] if prod.side[top] else live[top])
    top_ach = top_bytes / (top_ms * 1e-3) / 1e9
    alg = algorithmic_bytes(prod.A_h, prod.B_h, prod.products, prod.nnz, w)
    num_ms = float(np.median(res["num"]))
    achieved = alg / (num_ms * 1e-3) / 1e9
    traffic, tsrc = measured_traffic(top, top_bytes, args, workload, accumulator)
    roof = {"bound": "hbm", "achieved": round(top_ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(top_ach / peak, 4), "traffic": traffic, "traffic_source": tsrc,
            "kernel": f"numeric bin {top} ({BIN_NAMES[top]})", "ms": round(top_ms, 4),
            "ms_source": "serialised pass" if prod.side[top] else "bench steps (caller's stream)",
            "algorithmic_bytes": int(top_bytes), "peak_kind": peak_kind,
            "numeric_pass": {"achieved": round(achieved, 1), "frac": round(achieved / peak, 4),
                             "ms": round(num_ms, 4), "algorithmic_bytes": int(alg)}}
    per_bin = {BIN_NAMES[b]: {"ms_alone": round(float(serial[b]), 4), "cols": st["count"][b],
                              "products": st["products"][b], "nnz": st["nnz"][b],
                              "GBps_alone": round(bin_bytes(st, b, w) / (serial[b] * 1e-3) / 1e9, 1)
                              if serial[b] > 0 else None,
                              "stream_in_steps": "side" if prod.side[b] else "caller"}
               for b in range(1, len(serial)) if st["count"][b]}
    return roof, per_bin


def time_single_pass(A_h, B_h, dev, cfg, steps, warmup, flush):
    """Steps of the single-pass form through the C ABI (spgemm_single_pass,
    then spgemm_single_pass_copy into C), the workspace sized once
    beforehand (sizing depends only on the patterns, as allocation does)."""
    import torch
    from paper_2303_02471_gb300 import _native as N
    from paper_2303_02471_gb300 import ops
    A = ops.CscMatrix.from_host(A_h, device=dev)
    B = A if B_h is A_h else ops.CscMatrix.from_host(B_h, device=dev)
    hd = ops.handle(dev)
    lib = N.lib()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    cA, cB = ops._csc(A), ops._csc(B)
    ncfg = cfg.native()
    need = ops.single_pass_workspace_size(A, B, cfg, hd)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    colptr = torch.empty(B.ncols + 1, dtype=torch.int64, device=dev)

    def run():
        nnz, h = ctypes.c_int64(), ctypes.c_void_p()
        N.check(lib.spgemm_single_pass(hd.ptr, ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(ncfg),
                                       ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       ctypes.c_void_p(colptr.data_ptr()), ctypes.byref(nnz), ctypes.byref(h), sp),
                "spgemm_single_pass")
        return h, nnz.value

    h, nnz = run()
    lib.spg_plan_destroy(h)
    rows = torch.empty(nnz, dtype=torch.int32, device=dev)
    vals = torch.empty(nnz, dtype=A.dtype, device=dev)

    def copy(h):
        N.check(lib.spgemm_single_pass_copy(h, ctypes.c_void_p(colptr.data_ptr()), ctypes.c_void_p(rows.data_ptr()),
                                            ctypes.c_void_p(vals.data_ptr()), sp), "spgemm_single_pass_copy")

    for _ in range(warmup):
        h, _ = run()
        copy(h)
        lib.spg_plan_destroy(h)
    torch.cuda.synchronize()
    t_all, t_sp, t_cp = [], [], []
    for i in range(steps):
        flush.fill_(i & 0xff)
        ev = _events(3)
        ev[0].record(stream)
        h, _ = run()
        ev[1].record(stream)
        copy(h)
        ev[2].record(stream)
        N.check(lib.spg_plan_check(h, sp), "spg_plan_check")
        lib.spg_plan_destroy(h)
        t_all.append(ev[0].elapsed_time(ev[2]))
        t_sp.append(ev[0].elapsed_time(ev[1]))
        t_cp.append(ev[1].elapsed_time(ev[2]))
    return {"ms_per_step": round(float(np.median(t_all)), 4), "ms_single_pass": round(float(np.median(t_sp)), 4),
            "ms_copy": round(float(np.median(t_cp)), 4), "workspace_bytes": int(need)}


def measure_workload(k, args, dev, flush, steps, warmup, peak, peak_kind, cfg=None):
    """Steps, roofline and per-bin figures of workload k (a side entry)."""
    from paper_2303_02471_gb300 import ops
    A_h, B_h = make_workload(k)
    cfg = cfg or ops.Config()
    prod = Product(A_h, B_h, dev, cfg)
    res = time_steps(prod, steps, warmup, flush)
    serial = serial_bin_times(A_h, B_h, dev, cfg, flush)
    roof, per_bin = product_report(prod, res, serial, peak, peak_kind, None, workload=k,
                                   accumulator=cfg.small_accumulator)
    ms = float(np.median(res["step"]))
    out = {"workload": WORKLOADS[k], "products": int(prod.products), "nnz_C": int(prod.nnz), "t": prod.t,
           "value": round(2.0 * prod.products / (ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
           "ms_per_step": round(ms, 4),
           "phases_ms": {"symbolic": round(float(np.median(res["sym"])), 4),
                         "numeric": round(float(np.median(res["num"])), 4)},
           "roofline": roof, "numeric_bins": per_bin, "launches_per_step": prod.launches}
    sp = time_single_pass(A_h, B_h, dev, cfg, steps, warmup, flush)
    sp["value"] = round(2.0 * prod.products / (sp["ms_per_step"] * 1e-3) / 1e9, 3)
    sp["unit"] = "GFLOP/s"
    out["single_pass"] = sp
    del prod
    return out


def run_ours(args, rank, world):
    import torch
    from paper_2303_02471_gb300 import ops

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    A_h, B_h = make_workload(args.workload, args.rmat_scale)
    w = 8
    cfg = ops.Config(t=args.t, dense_cache_bytes=args.dense_cache, cta_threads=args.cta_threads,
                     small_accumulator=args.accumulator)
    prod = Product(A_h, B_h, dev, cfg)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    res = time_steps(prod, args.steps, args.warmup, flush, world, ClockSampler())
    ms = float(np.median(res["step"]))
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    products = prod.products
    value = world * 2.0 * products / (ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    serial = serial_bin_times(A_h, B_h, dev, cfg, flush)
    roof, per_bin = product_report(prod, res, serial, peak, peak_kind, args, w)

    # end to end through host buffers, right after the device-timed steps
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, A_h, B_h, products, prod, dev, world)
    sp_main = None
    if not args.no_aux:
        sp_main = time_single_pass(A_h, B_h, dev, cfg, max(3, min(args.steps, 10)), 3, flush)
        sp_main["value"] = round(2.0 * products / (sp_main["ms_per_step"] * 1e-3) / 1e9, 3)
        sp_main["unit"] = "GFLOP/s"

    line = None
    if rank == 0:
        base = None
        if not args.no_cpu_baseline and world == 1:
            base = cpu_baseline(A_h, B_h, args.cpu_seconds, "GFLOP/s")
        aux = {}
        if not args.no_aux:
            peak_w = (peak, peak_kind)
            others = {}
            for k in (2, 3):
                if k != args.workload:
                    others[str(k)] = measure_workload(k, args, dev, flush, max(3, min(args.steps, 10)), 3, *peak_w)
            # the light columns with hash tables in both phases (Section 3.2)
            # and with ESC in both phases (Section 4), beside the default
            # (ESC values, ESC counts in the bins of Op_j <= 64, hash-table
            # counts in the larger ones)
            ksteps = max(3, min(args.steps, 10))
            for k in (2, 3):
                entry = others.setdefault(str(k), {})
                for acc in ("hash", "esc"):
                    entry[acc] = measure_workload(k, args, dev, flush, ksteps, 3, *peak_w,
                                                  cfg=ops.Config(small_accumulator=acc))
            aux = {"workloads": others, "batched": run_batched(args, dev, *peak_w),
                   "backward": run_backward(args, dev, *peak_w),
                   "shards": run_shards(A_h, B_h, dev, flush, ms, prod)}
            if not args.no_sweep:
                aux["t_sweep"] = run_t_sweep(args, dev, flush)
        line = {"metric": METRIC, "value": round(value, 3),
                "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms, 4), "ms_per_step_mean": round(float(np.mean(res["step"])), 4),
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args), "t": prod.t, "products": int(products),
                           "nnz_C": int(prod.nnz), "l2": "512 MiB buffer written between timed steps",
                           "timing": "median of per-step CUDA events",
                           "parallelism": f"replicas x{world}"},
                "phases_ms": {"symbolic": round(float(np.median(res["sym"])), 4),
                              "numeric": round(float(np.median(res["num"])), 4)},
                "roofline": roof, "numeric_bins": per_bin, "single_pass": sp_main, "cpu_baseline": base, "e2e": e2e,
                **aux,
                "gpu_launches": prod.launches * args.steps,
                "clocks": res["clocks"]}
    return line


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def run_batched(args, dev, peak, peak_kind, count=512, fixed=None):
    """The 512-product batch: autotuned persistent launches (symbolic + numeric,
    numeric replayed from a CUDA graph) against the plain per-matrix calls
    through the C ABI with preallocated workspaces and outputs.  `count`
    takes the first products of the seeded batch; `fixed` (a Config) skips the
    tuner."""
    import torch
    from paper_2303_02471_gb300 import _native as N
    from paper_2303_02471_gb300 import autotune, ops, synth
    pairs = synth.batch_pairs(512, seed=0)[:count]
    As = [ops.CscMatrix.from_host(A, device=dev) for A, _ in pairs]
    Bs = [ops.CscMatrix.from_host(B, device=dev) for _, B in pairs]
    products = int(sum(A.ncols * (A.colptr[1] - A.colptr[0]) ** 2 for A, _ in pairs))
    if fixed is not None:
        cfg, rep = fixed, {"config": {"t": fixed.t, "hash_cta_max": fixed.hash_cta_max,
                                      "cta_threads": fixed.cta_threads}}
    else:
        cfg, rep = autotune.tune(As, Bs, repeats=1)
    side = torch.cuda.Stream(device=dev)
    steps = max(3, min(args.steps, 10))
    lib = N.lib()
    hd = ops.handle(dev)
    with torch.cuda.stream(side):
        plan = ops.spgemm_batched_symbolic(As, Bs, cfg)
        ops.spgemm_batched_numeric(plan, As, Bs, use_graph=True)
        ops.spgemm_batched_numeric(plan, As, Bs, use_graph=True)
        plan.check()
        ms = []
        for _ in range(steps):
            ev = _events(2)
            ev[0].record(side)
            ops.spgemm_batched_numeric(plan, As, Bs, use_graph=True)
            ev[1].record(side)
            side.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        num_ms = float(np.median(ms))
        ms = []
        for _ in range(steps):
            ev = _events(2)
            ev[0].record(side)
            p2 = ops.spgemm_batched_symbolic(As, Bs, cfg)
            ops.spgemm_batched_numeric(p2, As, Bs)
            ev[1].record(side)
            side.synchronize()
            p2.destroy()
            ms.append(ev[0].elapsed_time(ev[1]))
        step_ms = float(np.median(ms))
        plan.check()
        nnzs = plan.nnz
        # the plain per-matrix calls through the C ABI, every buffer allocated
        # beforehand: per product a symbolic call (it synchronises to read
        # nnz back) and a numeric call
        sp = ctypes.c_void_p(side.cuda_stream)
        prep = []
        for A, B, n in zip(As, Bs, nnzs):
            cA, cB = ops._csc(A), ops._csc(B)
            ncfg = cfg.native()
            ws = torch.empty(ops.workspace_size(A, B, cfg), dtype=torch.uint8, device=dev)
            cp = torch.empty(B.ncols + 1, dtype=torch.int64, device=dev)
            row = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
            val = torch.empty(max(n, 1), dtype=A.dtype, device=dev)
            prep.append((cA, cB, ncfg, ws, cp, row, val))

        def plain_symbolic(x):
            cA, cB, ncfg, ws, cp, row, val = x
            nnz, h = ctypes.c_int64(), ctypes.c_void_p()
            N.check(lib.spgemm_symbolic(hd.ptr, ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(ncfg),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(cp.data_ptr()),
                                        ctypes.byref(nnz), ctypes.byref(h), sp), "spgemm_symbolic")
            return h

        def plain_numeric(x, h):
            cA, cB, ncfg, ws, cp, row, val = x
            N.check(lib.spgemm_numeric(h, ctypes.byref(cA), ctypes.byref(cB), ctypes.c_void_p(cp.data_ptr()),
                                       ctypes.c_void_p(row.data_ptr()), ctypes.c_void_p(val.data_ptr()), sp),
                    "spgemm_numeric")

        for x in prep[:8]:
            h = plain_symbolic(x)
            plain_numeric(x, h)
            lib.spg_plan_destroy(h)
        side.synchronize()
        ev = _events(2)
        ev[0].record(side)
        for x in prep:
            h = plain_symbolic(x)
            plain_numeric(x, h)
            lib.spg_plan_destroy(h)
        ev[1].record(side)
        side.synchronize()
        plain_ms = ev[0].elapsed_time(ev[1])
        # the plain numeric calls alone, the plans made beforehand (the same
        # work as the batched numeric launch, one launch set per product)
        hs = [plain_symbolic(x) for x in prep]
        side.synchronize()
        ev = _events(2)
        ev[0].record(side)
        for x, h in zip(prep, hs):
            plain_numeric(x, h)
        ev[1].record(side)
        side.synchronize()
        plain_num_ms = ev[0].elapsed_time(ev[1])
        for h in hs:
            N.check(lib.spg_plan_check(h, sp), "spg_plan_check")
            lib.spg_plan_destroy(h)
        del prep
    launches = plan.info()["launches"]
    alg = sum(algorithmic_bytes(A, B, A.ncols * (A.colptr[1] - A.colptr[0]) ** 2, n,
                                8 if A.values.dtype == np.float64 else 4)
              for (A, B), n in zip(pairs, nnzs))
    ach = alg / (num_ms * 1e-3) / 1e9
    gf = lambda ms: round(2.0 * products / (ms * 1e-3) / 1e9, 3)
    return {"workload": "512 products C_i = A_i x B_i, n_i log-uniform 500..20000, Z_i ~ U{2..40}, "
                        "half f64 half f32", "products": products, "nnz_C": int(sum(nnzs)),
            "config": rep["config"], "GFLOPs_batched_step": gf(step_ms), "ms_batched_step": round(step_ms, 3),
            "GFLOPs_batched_numeric_graph": gf(num_ms), "ms_batched_numeric_graph": round(num_ms, 3),
            "GFLOPs_plain_per_matrix": gf(plain_ms), "ms_plain_per_matrix": round(plain_ms, 3),
            "GFLOPs_plain_numeric_only": gf(plain_num_ms), "ms_plain_numeric_only": round(plain_num_ms, 3),
            "plain": f"{count} x (spgemm_symbolic + spgemm_numeric) through the C ABI, buffers preallocated",
            "roofline": {"bound": "hbm", "kernel": "k_batched numeric (one persistent launch, graph replay)",
                         "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                         "algorithmic_bytes": int(alg), "ms": round(num_ms, 4), "peak_kind": peak_kind},
            "launches_symbolic_numeric": launches[:2]}


def run_shards(A_h, B_h, dev, flush, whole_ms, prod):
    """Column shards of the headline product (the columns of C are
    independent, Section 2.1): B cut into 2, 4 and 8 column blocks of about
    equal sum of Op_j (shard.column_ranges), each block's product (A
    replicated) timed on this GPU as a whole step.  The slowest block bounds a
    run of that many GPUs, one block each, with no collective; `balance` is
    the mean block time over the slowest."""
    from paper_2303_02471_gb300 import ops, shard
    plan = prod.plan()
    op = plan.op_counts().cpu().numpy()
    plan.destroy()
    out = {}
    for world in (2, 4, 8):
        ms = []
        for s, e in shard.column_ranges(op, world):
            blk = Product(A_h, shard.column_block(B_h, s, e), dev, ops.Config())
            res = time_steps(blk, 3, 1, flush, bin_timing=False)
            ms.append(float(np.median(res["step"])))
            del blk
        mx = max(ms)
        out[str(world)] = {"ms_per_block": [round(x, 4) for x in ms], "ms_slowest": round(mx, 4),
                           "ms_sum": round(sum(ms), 4), "speedup_bound": round(whole_ms / mx, 3),
                           "balance": round(float(np.mean(ms)) / mx, 3)}
    out["whole_ms"] = round(whole_ms, 4)
    return out


def run_backward(args, dev, peak, peak_kind):
    """Galerkin product P^T (A P) on the 40^3 Laplacian: forward (two products
    and the transpose) against the backward (two masked-product passes)."""
    import torch
    from paper_2303_02471_gb300 import ops, synth
    A_h, P_h = synth.workload(5)
    A = ops.CscMatrix.from_host(A_h, device=dev)
    P = ops.CscMatrix.from_host(P_h, device=dev)
    stream = torch.cuda.current_stream()

    def forward():
        M, pm = ops.spgemm(A, P)
        Pt, perm = ops.csc_transpose(P)
        C, pc = ops.spgemm(Pt, M)
        return M, pm, Pt, C, pc

    M, pm, Pt, C, pc = forward()
    G = torch.ones_like(C.values)
    products = pm.info()["products"] + pc.info()["products"]

    def backward():
        dPt, dM = ops.spgemm_backward(pc, Pt, M, C, G)
        _, dP = ops.spgemm_backward(pm, A, P, M, dM, need_dA=False)
        return dP

    for _ in range(3):
        forward()
        backward()
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 20))
    fw, bw = [], []
    for _ in range(steps):
        ev = _events(4)
        ev[0].record(stream)
        forward()
        ev[1].record(stream)
        ev[2].record(stream)
        backward()
        ev[3].record(stream)
        torch.cuda.synchronize()
        fw.append(ev[0].elapsed_time(ev[1]))
        bw.append(ev[2].elapsed_time(ev[3]))
    f_ms, b_ms = float(np.median(fw)), float(np.median(bw))
    Mh, Pth = M.to_host(), Pt.to_host()
    alg = (backward_bytes(Pth, Mh, pc.info()["products"], C.nnz, 8)
           + backward_bytes(A_h, P_h, pm.info()["products"], M.nnz, 8, need_dA=False))
    ach = alg / (b_ms * 1e-3) / 1e9
    gf = lambda ms: round(2.0 * products / (ms * 1e-3) / 1e9, 3)
    return {"workload": "Galerkin P^T (A P), A 40^3 7-point Laplacian, P 64000 x 8000 aggregation",
            "products": int(products), "ms_forward": round(f_ms, 4), "ms_backward": round(b_ms, 4),
            "GFLOPs_forward": gf(f_ms), "GFLOPs_backward": gf(b_ms),
            "forward": "two spgemm calls (symbolic + numeric, synchronising) and the transpose of P",
            "roofline_backward": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                                  "frac": round(ach / peak, 4), "algorithmic_bytes": int(alg),
                                  "ms": round(b_ms, 4), "peak_kind": peak_kind,
                                  "note": "about 1.2M products: launch-bound, not bandwidth-bound"}}


def run_t_sweep(args, dev, flush):
    """GFLOP/s of a whole step for t in SWEEP_T and the library's default t,
    on the random 2^20 product and the R-MAT 2^18 product; and of a batched
    step (symbolic + numeric) on the 512-product batch for the same t and the
    autotuner's choice; with the speed-up over t = 0 (every column in the
    dense SPA, Section 3.3)."""
    import torch
    from paper_2303_02471_gb300 import autotune, ops, synth
    out = {}
    for k in (2, 3):
        A_h, B_h = make_workload(k)
        row = {}
        for t in SWEEP_T + [None]:
            prod = Product(A_h, B_h, dev, ops.Config(t=t))
            res = time_steps(prod, 3, 1, flush, bin_timing=False)
            ms = float(np.median(res["step"]))
            key = "inf" if t == INF else ("default(%d)" % prod.t if t is None else str(t))
            row[key] = round(2.0 * prod.products / (ms * 1e-3) / 1e9, 3)
            del prod
        # the product autotuner's pick (t, table limit, CTA size, light-column accumulator)
        dA = ops.CscMatrix.from_host(A_h, device=dev)
        dB = dA if B_h is A_h else ops.CscMatrix.from_host(B_h, device=dev)
        tuned, rep = autotune.tune_product(dA, dB, repeats=1)
        del dA, dB
        prod = Product(A_h, B_h, dev, tuned)
        form = rep.get("form", "two_pass")
        if form == "single_pass":
            ms_t = time_single_pass(A_h, B_h, dev, tuned, 3, 1, flush)["ms_per_step"]
        else:
            ms_t = float(np.median(time_steps(prod, 3, 1, flush, bin_timing=False)["step"]))
        row["autotuned"] = round(2.0 * prod.products / (ms_t * 1e-3) / 1e9, 3)
        del prod
        base = row["0"]
        out[str(k)] = {"GFLOPs": row, "speedup_vs_t0": {k2: round(v / base, 3) for k2, v in row.items()},
                       "autotuned_config": {"t": tuned.t, "hash_cta_max": tuned.hash_cta_max,
                                            "cta_threads": tuned.cta_threads,
                                            "small_accumulator": tuned.small_accumulator,
                                            "table_slots_pct": tuned.table_slots_pct,
                                            "group_promote": tuned.group_promote, "form": form}}
    pairs = synth.batch_pairs(512, seed=0)
    As = [ops.CscMatrix.from_host(A, device=dev) for A, _ in pairs]
    Bs = [ops.CscMatrix.from_host(B, device=dev) for _, B in pairs]
    products = int(sum(A.ncols * (A.colptr[1] - A.colptr[0]) ** 2 for A, _ in pairs))
    tuned, _ = autotune.tune(As, Bs, repeats=1)
    row = {}
    stream = torch.cuda.current_stream()
    for name, cfg in [(("inf" if t == INF else str(t)), ops.Config(t=t)) for t in SWEEP_T] + [
            ("autotuned", tuned)]:
        try:
            ms = []
            for i in range(4):
                ev = _events(2)
                ev[0].record(stream)
                p = ops.spgemm_batched_symbolic(As, Bs, cfg)
                ops.spgemm_batched_numeric(p, As, Bs)
                ev[1].record(stream)
                torch.cuda.synchronize()
                p.destroy()
                if i:
                    ms.append(ev[0].elapsed_time(ev[1]))
            row[name] = round(2.0 * products / (float(np.median(ms)) * 1e-3) / 1e9, 3)
        except RuntimeError as e:  # a threshold the batched kernels do not take
            row[name] = str(e)
    base = row.get("0")
    out["4"] = {"GFLOPs": row, "speedup_vs_t0": {k2: round(v / base, 3) for k2, v in row.items()
                                                  if isinstance(v, float) and isinstance(base, float)},
                "autotuned_config": {"t": tuned.t, "hash_cta_max": tuned.hash_cta_max,
                                     "cta_threads": tuned.cta_threads, "table_slots_pct": tuned.table_slots_pct,
                                     "group_promote": tuned.group_promote}}
    return out


def run_e2e(args, A_h, B_h, products, prod, dev, world):
    """Same metric with host inputs and outputs, through the C ABI: every step
    copies its inputs from pinned host memory, runs both phases and reads C
    (colptr, rows, values) back into pinned host memory.  Steps are pipelined
    as a stream of products would be: the read-back of step i (its own
    stream, double-buffered outputs) overlaps the copy-in and compute of step
    i + 1.  The device-to-host link, not the kernels, bounds this number."""
    import torch
    from paper_2303_02471_gb300 import _native as N
    from paper_2303_02471_gb300 import ops
    lib, ncfg, cfg, hd = prod.lib, prod.ncfg, prod.cfg, prod.hd

    def pin(x):
        return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    hA = [pin(A_h.colptr), pin(A_h.rowidx.astype(np.int32)), pin(A_h.values)]
    same = B_h is A_h
    hB = hA if same else [pin(B_h.colptr), pin(B_h.rowidx.astype(np.int32)), pin(B_h.values)]
    dA = [torch.empty_like(x, device=dev) for x in hA]
    dB = dA if same else [torch.empty_like(x, device=dev) for x in hB]
    A = ops.CscMatrix(A_h.nrows, A_h.ncols, *dA)
    B = ops.CscMatrix(B_h.nrows, B_h.ncols, *dB)
    cA, cB = ops._csc(A), ops._csc(B)
    ws = torch.empty(ops.workspace_size(A, B, cfg), dtype=torch.uint8, device=dev)
    s_run, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    sp = ctypes.c_void_p(s_run.cuda_stream)
    h2d = sum(x.numel() * x.element_size() for x in hA) + (0 if same else sum(x.numel() * x.element_size() for x in hB))
    bufs = [{"colptr": torch.empty(B.ncols + 1, dtype=torch.int64, device=dev),
             "hcp": torch.empty(B.ncols + 1, dtype=torch.int64, pin_memory=True),
             "freed": None} for _ in range(2)]
    state = {"i": 0, "n": 0}

    def step():
        o = bufs[state["i"] % 2]
        state["i"] += 1
        with torch.cuda.stream(s_run):
            if o["freed"] is not None:  # the read-back two steps ago is done with these buffers
                s_run.wait_event(o["freed"])
            for d, hsrc in zip(dA, hA):
                d.copy_(hsrc, non_blocking=True)
            if not same:
                for d, hsrc in zip(dB, hB):
                    d.copy_(hsrc, non_blocking=True)
            nnz, h = ctypes.c_int64(), ctypes.c_void_p()
            N.check(lib.spgemm_symbolic(hd.ptr, ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(ncfg),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                        ctypes.c_void_p(o["colptr"].data_ptr()), ctypes.byref(nnz),
                                        ctypes.byref(h), sp), "spgemm_symbolic")
            n = nnz.value
            if "row" not in o or o["row"].numel() != n:
                o["row"] = torch.empty(n, dtype=torch.int32, device=dev)
                o["val"] = torch.empty(n, dtype=torch.float64, device=dev)
                o["hrow"] = torch.empty(n, dtype=torch.int32, pin_memory=True)
                o["hval"] = torch.empty(n, dtype=torch.float64, pin_memory=True)
            N.check(lib.spgemm_numeric(h, ctypes.byref(cA), ctypes.byref(cB),
                                       ctypes.c_void_p(o["colptr"].data_ptr()),
                                       ctypes.c_void_p(o["row"].data_ptr()),
                                       ctypes.c_void_p(o["val"].data_ptr()), sp), "spgemm_numeric")
            done = torch.cuda.Event()
            done.record(s_run)
            st = lib.spg_plan_check(h, sp)
            lib.spg_plan_destroy(h)
            N.check(st, "spg_plan_check")
        with torch.cuda.stream(s_out):
            s_out.wait_event(done)
            o["hcp"].copy_(o["colptr"], non_blocking=True)
            o["hrow"].copy_(o["row"], non_blocking=True)
            o["hval"].copy_(o["val"], non_blocking=True)
            o["freed"] = torch.cuda.Event()
            o["freed"].record(s_out)
        state["n"] = n
        return n

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    steps = max(2, min(args.steps, 10))
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0.record(s_run)
    for _ in range(steps):
        n = step()
    s_out.wait_stream(s_run)
    t1.record(s_out)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    if world > 1:
        torch.distributed.barrier()
        tm = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tm, op=torch.distributed.ReduceOp.MAX)
        ms = float(tm.item())
    # the last read-back landed: spot-check it against the device copy
    o = bufs[(state["i"] - 1) % 2]
    assert torch.equal(o["hrow"][:: 1 << 16], o["row"][:: 1 << 16].cpu())
    d2h = 8 * (B.ncols + 1) + n * 12
    return {"value": round(world * 2.0 * products / (ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": round(ms, 3), "steps": steps, "pipelined": True,
            "d2h_GBps": round(d2h / (ms * 1e-3) / 1e9, 1)}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.batched_only > 0:
        from paper_2303_02471_gb300 import ops
        peak, kind = peaks()
        line = {"batched": run_batched(args, "cuda:0", peak, kind, count=args.batched_only,
                                       fixed=ops.Config(t=33, hash_cta_max=8192, cta_threads=128))}
    else:
        line = run_ours(args, rank, world)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

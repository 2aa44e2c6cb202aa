"""Benchmark of the GB300 column-wise SpGEMM (one JSON line on rank 0).

A step is one pass of the whole hot path over the workload: input
validation, Op_j and binning, symbolic pass, scan, numeric pass with sorted
output (spgemm_symbolic + spgemm_numeric through the C ABI).  Default
workload: C = A x A with A an R-MAT power-law matrix (2^18 rows, a,b,c,d =
0.57,0.19,0.19,0.05, 8 edges per row drawn, columns capped at 2000 entries,
FP64 values U[-1,1]), the largest single product of the workload set.

Metric: GFLOP/s = 2 x sum_j Op_j / step time (Op_j = products of column j).
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


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", type=int, default=3, choices=[1, 2, 3])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-aux", action="store_true",
                   help="skip the batched (512 products) and backward (Galerkin 40^3) measurements")
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
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# DRAM bytes (read + write) of one launch of the dominant kernel, R-MAT 2^18
# default configuration, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum, 1 pass; profiles/k_num_dense_rmat18_traffic.md).
# Valid only for the kernel sources it was taken with: the hash below covers
# the files that define that kernel, and any change there reports null.
MEASURED_TRAFFIC = {"bin": 13, "scale": 18, "bytes": 2.12e9 + 6.43e9, "sources_sha256_16": "364fef5be9c87077",
                    "sources": ("spgemm_internal.cuh", "kernels.cuh", "columns.cuh", "numeric.cu")}


def measured_traffic(top_bin, args):
    import hashlib
    t = MEASURED_TRAFFIC
    default_cfg = args.t is None and args.cta_threads is None and args.dense_cache is None
    if args.workload != 3 or args.rmat_scale != t["scale"] or top_bin != t["bin"] or not default_cfg:
        return None
    h = hashlib.sha256()
    root = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2303_02471_gb300", "csrc")
    for f in t["sources"]:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    return int(t["bytes"]) if h.hexdigest()[:16] == t["sources_sha256_16"] else None


def algorithmic_bytes(A, B, products, nnzC, w):
    """Numeric pass, per launch: B columns (colptr, rows, values), the
    gathered A column pointers and A entries of every product, and C written
    once (colptr read, rows and values written)."""
    nB = B.ncols
    nnzB = int(B.colptr[-1])
    return (8 * (nB + 1) + nnzB * (4 + w) + 16 * nnzB + products * (4 + w)
            + 8 * (nB + 1) + nnzC * (4 + w))


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


def cpu_baseline(A, B, target_s, unit):
    """The oracle as it stands, on a bounded column sample, all host cores."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    op = oracle.op_counts(A, B)
    threads = oracle.threads(cores)
    # estimate the rate on a small sample, then size the timed one
    small, cols = column_sample(B, 0.005, seed=1)
    t0 = time.perf_counter()
    oracle.spgemm(A, small, nthreads=threads)
    rate = max(1.0, op[cols].sum()) / max(1e-3, time.perf_counter() - t0)
    frac = min(1.0, target_s * rate / max(1, op.sum()))
    sample, cols = column_sample(B, frac, seed=2)
    products = int(op[cols].sum())
    t0 = time.perf_counter()
    oracle.spgemm(A, sample, nthreads=threads)
    dt = time.perf_counter() - t0
    return {"value": 2.0 * products / dt / 1e9, "unit": unit, "cores": threads, "kind": "oracle",
            "sample": f"{len(cols)} of {B.ncols} columns of B (seeded, p={frac:.4f}), "
                      f"{products} products, {dt:.2f} s"}


# ------------------------------------------------------------------ arms
REFERENCE_BUDGET_S = 60.0  # host seconds of the whole reference run


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores, as the other arm: W untimed
    and K timed steps, every step the same seeded column sample of the
    workload, sized so that the whole run takes about a minute."""
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
    frac = min(1.0, per_step * rate / max(1, op.sum()))
    sample, cols = column_sample(B, frac, seed=2)
    products = int(op[cols].sum())
    for _ in range(args.warmup):
        oracle.spgemm(A, sample, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spgemm(A, sample, nthreads=threads)
    dt = time.perf_counter() - t0
    value = 2.0 * products * args.steps / dt / 1e9
    base = {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
            "sample": f"{len(cols)} of {B.ncols} columns of B per step (seeded, p={frac:.4f}), "
                      f"{products} products, {args.steps} timed steps in {dt:.2f} s"}
    return {"impl": "reference", "metric": "SpGEMM GFLOP/s (2 x intermediate products / s)",
            "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / max(1, args.steps), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args)},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_ours(args, rank, world):
    import torch
    from paper_2303_02471_gb300 import _native as N
    from paper_2303_02471_gb300 import ops

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    A_h, B_h = make_workload(args.workload, args.rmat_scale)
    w = 8
    A = ops.CscMatrix.from_host(A_h, device=dev)
    B = A if B_h is A_h else ops.CscMatrix.from_host(B_h, device=dev)
    cfg = ops.Config(t=args.t, dense_cache_bytes=args.dense_cache, cta_threads=args.cta_threads)
    ncfg = cfg.native()
    lib = N.lib()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    cA, cB = ops._csc(A), ops._csc(B)
    ws = torch.empty(ops.workspace_size(A, B, cfg), dtype=torch.uint8, device=dev)
    colptr = torch.empty(B.ncols + 1, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def symbolic():
        nnz, h = ctypes.c_int64(), ctypes.c_void_p()
        N.check(lib.spgemm_symbolic(ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(ncfg),
                                    ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                    ctypes.c_void_p(colptr.data_ptr()), ctypes.byref(nnz),
                                    ctypes.byref(h), sp), "spgemm_symbolic")
        return h, nnz.value

    h, nnz = symbolic()
    first = ops.Plan(h, ws, A, B, colptr, nnz, cfg)
    info = first.info()
    st = first.bin_stats()
    st["count"] = info["bins"]
    products = info["products"]
    lc = first.launch_count()
    launches_per_step = lc["symbolic"] + lc["numeric"]
    first.destroy()
    rowidx = torch.empty(nnz, dtype=torch.int32, device=dev)
    values = torch.empty(nnz, dtype=torch.float64, device=dev)

    def numeric(plan):
        N.check(lib.spgemm_numeric(plan.handle, ctypes.byref(cA), ctypes.byref(cB),
                                   ctypes.c_void_p(colptr.data_ptr()),
                                   ctypes.c_void_p(rowidx.data_ptr()),
                                   ctypes.c_void_p(values.data_ptr()), sp), "spgemm_numeric")

    def plan_of(hh, n):
        return ops.Plan(hh, ws, A, B, colptr, n, cfg)

    for _ in range(args.warmup):
        plan = plan_of(*symbolic())
        numeric(plan)
        plan.check()
        plan.destroy()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    bin_ms = []
    clocks = ClockSampler()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(i & 0xff)  # evict A and B from L2 between steps
        ev[i][0].record(stream)
        plan = plan_of(*symbolic())
        plan.set_timing(True)
        ev[i][1].record(stream)
        numeric(plan)
        ev[i][2].record(stream)
        plan.check()
        bin_ms.append(plan.bin_times())
        plan.destroy()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    num_ms = [b.elapsed_time(c) for a, b, c in ev]
    ms = float(np.mean(step_ms))
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = world * 2.0 * products / (ms * 1e-3) / 1e9

    # roofline: the dominant kernel (the bin kernel with the most algorithmic
    # bytes) and the whole binned numeric pass.  Beside a dense bin the
    # lane-group bins run on side streams: their event times start with the
    # pass and include waiting for SMs, so they do not pick the kernel.
    peak, peak_kind = peaks()
    bms = np.mean(np.array(bin_ms), axis=0)
    top = dominant_bin(st, w)
    side = bool(st["count"][13]) and any(st["count"][b] for b in range(1, 7))
    top_bytes = bin_bytes(st, top, w)
    top_ach = top_bytes / (bms[top] * 1e-3) / 1e9
    alg = algorithmic_bytes(A_h, B_h, products, nnz, w)
    num_avg = float(np.mean(num_ms))
    achieved = alg / (num_avg * 1e-3) / 1e9
    names = ["empty"] + [f"hash_group_op<={o}" for o in (8, 16, 32, 64, 128, 256)] + \
        [f"hash_cta_op<={o}" for o in (512, 1024, 2048, 4096, 8192)] + ["hash_global", "dense_spa"]
    roof = {"bound": "hbm", "achieved": round(top_ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(top_ach / peak, 4), "traffic": measured_traffic(top, args),
            "kernel": f"numeric bin {top} ({names[top]})", "ms": round(float(bms[top]), 4),
            "algorithmic_bytes": int(top_bytes), "peak_kind": peak_kind,
            "numeric_pass": {"achieved": round(achieved, 1), "frac": round(achieved / peak, 4),
                             "ms": round(num_avg, 4), "algorithmic_bytes": int(alg)}}
    per_bin = {names[b]: {"ms": round(float(bms[b]), 4), "cols": st["count"][b],
                          "products": st["products"][b], "nnz": st["nnz"][b],
                          "GBps": round(bin_bytes(st, b, w) / (bms[b] * 1e-3) / 1e9, 1),
                          "stream": "side" if side and 1 <= b <= 6 else "caller"}
               for b in range(1, len(bms)) if st["count"][b]}

    # end to end through host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, A_h, B_h, products, lib, ncfg, cfg, dev, stream, world)

    line = None
    if rank == 0:
        base = None
        if not args.no_cpu_baseline and world == 1:
            base = cpu_baseline(A_h, B_h, args.cpu_seconds, "GFLOP/s")
        aux = {}
        if not args.no_aux:
            aux = {"batched": run_batched(args, dev), "backward": run_backward(args, dev)}
        line = {"metric": "SpGEMM GFLOP/s (2 x intermediate products / s)", "value": round(value, 3),
                "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args), "t": info["t"], "products": int(products),
                           "nnz_C": int(nnz), "l2": "512 MiB buffer written between timed steps",
                           "parallelism": f"replicas x{world}"},
                "phases_ms": {"symbolic": round(float(np.mean([a.elapsed_time(b) for a, b, c in ev])), 4),
                              "numeric": round(num_avg, 4)},
                "roofline": roof, "numeric_bins": per_bin, "cpu_baseline": base, "e2e": e2e, **aux,
                "gpu_launches": launches_per_step * args.steps,
                "clocks": clk}
    return line


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def run_batched(args, dev):
    """The 512-product batch: autotuned persistent launches (symbolic + numeric,
    numeric replayed from a CUDA graph) against the plain per-matrix calls."""
    import torch
    from paper_2303_02471_gb300 import autotune, ops, synth
    pairs = synth.batch_pairs(512, seed=0)
    As = [ops.CscMatrix.from_host(A, device=dev) for A, _ in pairs]
    Bs = [ops.CscMatrix.from_host(B, device=dev) for _, B in pairs]
    products = int(sum(A.ncols * (A.colptr[1] - A.colptr[0]) ** 2 for A, _ in pairs))
    cfg, rep = autotune.tune(As, Bs, repeats=1)
    side = torch.cuda.Stream(device=dev)
    steps = max(3, min(args.steps, 10))
    with torch.cuda.stream(side):
        plan = ops.spgemm_batched_symbolic(As, Bs, cfg)
        ops.spgemm_batched_numeric(plan, As, Bs, use_graph=True)
        ops.spgemm_batched_numeric(plan, As, Bs, use_graph=True)
        plan.check()
        ev = _events(2)
        ev[0].record(side)
        for _ in range(steps):
            ops.spgemm_batched_numeric(plan, As, Bs, use_graph=True)
        ev[1].record(side)
        side.synchronize()
        num_ms = ev[0].elapsed_time(ev[1]) / steps
        ev = _events(2)
        ev[0].record(side)
        for _ in range(steps):
            p2 = ops.spgemm_batched_symbolic(As, Bs, cfg)
            ops.spgemm_batched_numeric(p2, As, Bs)
            p2.destroy()
        ev[1].record(side)
        side.synchronize()
        step_ms = ev[0].elapsed_time(ev[1]) / steps
        plan.check()
        # plain per-matrix calls, same products
        for A, B in zip(As[:8], Bs[:8]):
            ops.spgemm(A, B, cfg)
        ev = _events(2)
        ev[0].record(side)
        for A, B in zip(As, Bs):
            C, pl = ops.spgemm(A, B, cfg)
            pl.destroy()
        ev[1].record(side)
        side.synchronize()
        plain_ms = ev[0].elapsed_time(ev[1])
    launches = plan.info()["launches"]
    gf = lambda ms: round(2.0 * products / (ms * 1e-3) / 1e9, 3)
    return {"workload": "512 products C_i = A_i x B_i, n_i log-uniform 500..20000, Z_i ~ U{2..40}, "
                        "half f64 half f32", "products": products,
            "config": rep["config"], "GFLOPs_batched_step": gf(step_ms), "ms_batched_step": round(step_ms, 3),
            "GFLOPs_batched_numeric_graph": gf(num_ms), "ms_batched_numeric_graph": round(num_ms, 3),
            "GFLOPs_plain_per_matrix": gf(plain_ms), "ms_plain_per_matrix": round(plain_ms, 3),
            "launches_symbolic_numeric": launches[:2]}


def run_backward(args, dev):
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
    ev = _events(4)
    ev[0].record(stream)
    for _ in range(steps):
        forward()
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(steps):
        backward()
    ev[3].record(stream)
    torch.cuda.synchronize()
    f_ms = ev[0].elapsed_time(ev[1]) / steps
    b_ms = ev[2].elapsed_time(ev[3]) / steps
    gf = lambda ms: round(2.0 * products / (ms * 1e-3) / 1e9, 3)
    return {"workload": "Galerkin P^T (A P), A 40^3 7-point Laplacian, P 64000 x 8000 aggregation",
            "products": int(products), "ms_forward": round(f_ms, 4), "ms_backward": round(b_ms, 4),
            "GFLOPs_forward": gf(f_ms), "GFLOPs_backward": gf(b_ms)}


def run_e2e(args, A_h, B_h, products, lib, ncfg, cfg, dev, stream, world):
    """Same metric with host inputs and outputs, through the C ABI: every step
    copies its inputs from pinned host memory, runs both phases and reads C
    (colptr, rows, values) back into pinned host memory.  Steps are pipelined
    as a stream of products would be: the read-back of step i (its own
    stream, double-buffered outputs) overlaps the copy-in and compute of step
    i + 1.  The device-to-host link, not the kernels, bounds this number."""
    import torch
    from paper_2303_02471_gb300 import _native as N
    from paper_2303_02471_gb300 import ops

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
            N.check(lib.spgemm_symbolic(ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(ncfg),
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
    line = run_ours(args, rank, world)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Autotuners: for a batch (the H-HASH threshold t, the largest shared-memory
hash table hash_cta_max and the threads per CTA of the persistent kernels)
and for a single product (t, hash_cta_max, the threads per CTA of the CTA
bins and the accumulator of the light columns), each by timing candidate
configurations on the products themselves.  A second stage then tries, around
the best of the grid, the hash-table size (slots per output entry) and the
lanes per light column (how many lane-group bins a light column moves up):
the table sizes and threads per column of Section 3.2's hash accumulation.
For a single product a last stage times the pick in the single-pass form too
and reports the faster form (`form` in the report).

The paper fixes t = 40 for its vector unit and studies t, b_min and b_max by
hand (Section 5.4); here the choice is measured on the GPU and cached per GPU
model and batch signature (JSON under $XDG_CACHE_HOME/spgemm_gb300 or the
path given).
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
from typing import Optional

import numpy as np
import torch

from . import ops
from .ops import Config

INF = (1 << 63) - 1
DEFAULT_GRID = {
    "t": [33, 65, 129, 257, 513, 1025, None],
    "hash_cta_max": [2048, 8192],
    "cta_threads": [128, 256, 512],
}
# Knobs tried in the second stage, one combination at a time around the best
# configuration of the first (the first value of each is the library default).
REFINE = {
    "table_slots_pct": [150, 250],
    "group_promote": [0, 1],
}
# Forms of a single product tried last with the pick (grid key "form"): both
# phases, or the single pass (Op_j-sized slots, then a copy into C).
FORMS = ["two_pass", "single_pass"]


def _with_defaults(conf: dict, refine: dict) -> dict:
    """conf with the second stage's knobs spelled out (their first values,
    the library defaults, where the first stage's pick kept them)."""
    out = dict(conf)
    for n, values in refine.items():
        out.setdefault(n, values[0])
    return out


def _refine(best_conf: dict, timed, results: list, refine: dict) -> None:
    """Times best_conf with every combination of the refine values other than
    the defaults (appending to results)."""
    names = sorted(refine)
    for values in itertools.product(*(refine[n] for n in names)):
        conf = dict(best_conf)
        conf.update(zip(names, values))
        if all(v == refine[n][0] for n, v in zip(names, values)):
            continue  # the first stage timed the defaults
        try:
            ms, err = timed(conf), None
        except RuntimeError as e:  # a configuration the products do not support
            ms, err = float("inf"), str(e)
        results.append({"config": conf, "ms": ms, "error": err})


def _cache_path(path: Optional[str]) -> str:
    if path:
        return path
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "spgemm_gb300", "autotune.json")


def signature(As, Bs) -> str:
    """GPU model, batch size, dtype mix and log2 histograms of the sizes."""
    dev = torch.cuda.get_device_name(As[0].device) if As else "none"
    n = np.array([B.ncols for B in Bs], dtype=np.int64)
    z = np.array([B.nnz / max(1, B.ncols) for B in Bs])
    f64 = sum(1 for A in As if A.dtype == torch.float64)
    h = (np.bincount(np.log2(np.maximum(n, 1)).astype(int), minlength=32).tolist(),
         np.bincount(np.log2(np.maximum(z, 1)).astype(int), minlength=16).tolist())
    key = json.dumps([dev, len(As), f64, h])
    return hashlib.sha1(key.encode()).hexdigest()


def _time(As, Bs, cfg: Config, repeats: int) -> float:
    plan = ops.spgemm_batched_symbolic(As, Bs, cfg)
    ops.spgemm_batched_numeric(plan, As, Bs)
    plan.check()
    stream = torch.cuda.current_stream()
    best = float("inf")
    for _ in range(repeats):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        p = ops.spgemm_batched_symbolic(As, Bs, cfg)
        e1.record(stream)
        ops.spgemm_batched_numeric(p, As, Bs)
        e2.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e2))
        p.destroy()
    plan.destroy()
    return best


def tune(As, Bs, grid: Optional[dict] = None, repeats: int = 2, cache: Optional[str] = None,
         refresh: bool = False):
    """Best Config for the batch (cached).  Returns (config, report)."""
    path = _cache_path(cache)
    key = signature(As, Bs)
    table = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if key in table and not refresh:
        return Config(**table[key]["config"]), table[key]
    grid = grid or dict(DEFAULT_GRID, **REFINE)
    results = []
    for t, hmax, thr in itertools.product(grid["t"], grid["hash_cta_max"], grid["cta_threads"]):
        cfg = Config(t=t, hash_cta_max=hmax, cta_threads=thr)
        try:
            ms = _time(As, Bs, cfg, repeats)
        except RuntimeError as e:  # a shape the candidate does not support
            ms = float("inf")
            err = str(e)
        else:
            err = None
        results.append({"config": {"t": t, "hash_cta_max": hmax, "cta_threads": thr}, "ms": ms, "error": err})
    ok = [r for r in results if np.isfinite(r["ms"])]
    if not ok:
        raise RuntimeError("no candidate configuration ran")
    refine = {n: grid[n] for n in REFINE if n in grid}
    if refine:
        best = min(ok, key=lambda r: r["ms"])
        _refine(best["config"], lambda conf: _time(As, Bs, Config(**conf), repeats), results, refine)
        ok = [r for r in results if np.isfinite(r["ms"])]
    best = min(ok, key=lambda r: r["ms"])
    entry = {"config": _with_defaults(best["config"], refine), "ms": best["ms"], "candidates": results}
    table[key] = entry
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass
    return Config(**entry["config"]), entry


PRODUCT_GRID = {
    "t": [65, 129, 257, 513, 1025, None],
    "hash_cta_max": [2048, 8192],
    "cta_threads": [512, 1024],
    "small_accumulator": ["hash", "esc", "auto"],
}


def product_signature(A, B) -> str:
    """GPU model, shapes, nnz, dtype and log2 histograms of the column lengths
    of A and B (the quantities Op_j and the bins follow from)."""
    dev = torch.cuda.get_device_name(A.device)

    def hist(M):
        z = torch.diff(M.colptr).clamp(min=1).double().log2().floor().long().cpu().numpy()
        return np.bincount(z, minlength=32).tolist()
    key = json.dumps([dev, "product", A.nrows, A.ncols, B.ncols, A.nnz, B.nnz, str(A.dtype), hist(A), hist(B)])
    return hashlib.sha1(key.encode()).hexdigest()


def _time_product(A, B, cfg: Config, repeats: int) -> float:
    C, plan = ops.spgemm(A, B, cfg)
    plan.check()
    plan.destroy()
    stream = torch.cuda.current_stream()
    best = float("inf")
    for _ in range(repeats):
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(stream)
        _, _, p = ops.spgemm_symbolic(A, B, cfg)
        ops.spgemm_numeric(p, A, B, C.rowidx, C.values)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
        p.destroy()
    return best


def _time_single_pass(A, B, cfg: Config, repeats: int) -> float:
    ws = torch.empty(max(ops.single_pass_workspace_size(A, B, cfg), 256), dtype=torch.uint8, device=A.device)
    C, plan = ops.spgemm_single_pass(A, B, cfg, workspace=ws)
    plan.check()
    plan.destroy()
    del C
    stream = torch.cuda.current_stream()
    best = float("inf")
    for _ in range(repeats):
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(stream)
        C, p = ops.spgemm_single_pass(A, B, cfg, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
        p.destroy()
        del C
    return best


def tune_product(A, B, grid: Optional[dict] = None, repeats: int = 2, cache: Optional[str] = None,
                 refresh: bool = False):
    """Best Config for one product C = A B, timed as a whole step (symbolic
    and numeric phases) per candidate; cached per GPU model and pattern
    signature.  Returns (config, report)."""
    path = _cache_path(cache)
    key = product_signature(A, B)
    table = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if key in table and not refresh:
        return Config(**table[key]["config"]), table[key]
    grid = grid or dict(PRODUCT_GRID, **REFINE, form=FORMS)
    refine = {n: grid[n] for n in REFINE if n in grid}
    forms = grid.get("form", [])
    names = sorted(n for n in grid if n not in refine and n != "form")
    results = []
    for values in itertools.product(*(grid[n] for n in names)):
        conf = dict(zip(names, values))
        try:
            ms = _time_product(A, B, Config(**conf), repeats)
            err = None
        except RuntimeError as e:  # a configuration the product does not support
            ms, err = float("inf"), str(e)
        results.append({"config": conf, "ms": ms, "error": err})
    ok = [r for r in results if np.isfinite(r["ms"])]
    if not ok:
        raise RuntimeError("no candidate configuration ran")
    if refine:
        best = min(ok, key=lambda r: r["ms"])
        _refine(best["config"], lambda conf: _time_product(A, B, Config(**conf), repeats), results, refine)
        ok = [r for r in results if np.isfinite(r["ms"])]
    best = min(ok, key=lambda r: r["ms"])
    form, best_ms = "two_pass", best["ms"]
    if "single_pass" in forms:
        # the pick's configuration in the single pass (whole call, copy included)
        try:
            ms, err = _time_single_pass(A, B, Config(**best["config"]), repeats), None
        except RuntimeError as e:
            ms, err = float("inf"), str(e)
        results.append({"config": dict(best["config"], form="single_pass"), "ms": ms, "error": err})
        if ms < best_ms:
            form, best_ms = "single_pass", ms
    entry = {"config": _with_defaults(best["config"], refine), "form": form, "ms": best_ms, "candidates": results}
    table[key] = entry
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass
    return Config(**entry["config"]), entry

"""Partitioning for several GPUs (one process per GPU, no data-path collective).

The columns of C = A B are independent (Section 2.1 of arXiv 2303.02471):
rank r computes the column block C[:, c_r:c_{r+1}] = A B[:, c_r:c_{r+1}] from
a replicated A and its column range of B.  The ranges are cut so that every
rank gets about the same number of products (sum of Op_j).  For a batch of
independent products, whole products are dealt to ranks by estimated cost
(longest first, to the least loaded rank).  Only host logic lives here; the
products themselves run through the single-GPU calls on each rank.
"""
from __future__ import annotations

from types import SimpleNamespace
from typing import List, Sequence, Tuple

import numpy as np


def column_ranges(op: np.ndarray, world: int) -> List[Tuple[int, int]]:
    """[start, end) column ranges with about equal sum of Op_j per rank."""
    op = np.asarray(op, dtype=np.int64)
    n = op.shape[0]
    if world < 1:
        raise ValueError("world must be >= 1")
    cum = np.cumsum(op)
    total = int(cum[-1]) if n else 0
    cuts = [0]
    for r in range(1, world):
        c = int(np.searchsorted(cum, total * r / world, side="left")) if total else (n * r) // world
        cuts.append(min(max(c, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def column_block(M, start: int, end: int):
    """CSC of M's columns [start, end) (host arrays, shared row/value slices)."""
    lo, hi = int(M.colptr[start]), int(M.colptr[end])
    return SimpleNamespace(nrows=M.nrows, ncols=end - start,
                           colptr=np.asarray(M.colptr[start:end + 1], dtype=np.int64) - lo,
                           rowidx=M.rowidx[lo:hi], values=M.values[lo:hi])


def concat_columns(blocks: Sequence) -> SimpleNamespace:
    """Column blocks side by side (the inverse of column_block over ranges)."""
    nrows = blocks[0].nrows
    cps, rows, vals, off = [np.zeros(1, dtype=np.int64)], [], [], 0
    for b in blocks:
        cps.append(np.asarray(b.colptr[1:], dtype=np.int64) + off)
        off += int(b.colptr[-1])
        rows.append(np.asarray(b.rowidx))
        vals.append(np.asarray(b.values))
    return SimpleNamespace(nrows=nrows, ncols=sum(b.ncols for b in blocks), colptr=np.concatenate(cps),
                           rowidx=np.concatenate(rows), values=np.concatenate(vals))


def deal_products(costs: Sequence[int], world: int) -> List[List[int]]:
    """Product indices per rank: longest first, each to the least loaded rank."""
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-int(costs[k]), k)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += int(costs[i])
    for lst in out:
        lst.sort()
    return out

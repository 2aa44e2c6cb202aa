"""Multi-rank partitioning on CPU: two gloo ranks each compute a column block
(or a share of a batch) with the oracle; together they reproduce the whole."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2303_02471_gb300 import shard, synth


def test_column_ranges_balance_and_cover():
    A = synth.rmat(12, seed=3, col_cap=300)
    op = oracle.op_counts(A, A)
    for world in (1, 2, 3, 8):
        rs = shard.column_ranges(op, world)
        assert rs[0][0] == 0 and rs[-1][1] == A.ncols
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        loads = [int(op[s:e].sum()) for s, e in rs]
        assert max(loads) - min(loads) <= 2 * int(op.max())


def test_deal_products_covers_each_once():
    costs = [5, 1, 9, 3, 3, 7, 0, 2]
    parts = shard.deal_products(costs, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    A = synth.rmat(11, seed=9, col_cap=200)
    op = oracle.op_counts(A, A)
    s, e = shard.column_ranges(op, world)[rank]
    C, _ = oracle.spgemm(A, shard.column_block(A, s, e))
    # the data path needs no exchange; the gather only checks the result
    blocks = [None] * world
    dist.all_gather_object(blocks, (C.colptr, C.rowidx, C.values, C.nrows, C.ncols))
    if rank == 0:
        from types import SimpleNamespace
        parts = [SimpleNamespace(colptr=b[0], rowidx=b[1], values=b[2], nrows=b[3], ncols=b[4]) for b in blocks]
        full = shard.concat_columns(parts)
        ref, _ = oracle.spgemm(A, A)
        q.put(bool(np.array_equal(full.colptr, ref.colptr) and np.array_equal(full.rowidx, ref.rowidx)
                   and np.array_equal(full.values, ref.values)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_product():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True

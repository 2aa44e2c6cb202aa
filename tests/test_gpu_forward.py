"""Parity of the CUDA forward path (through the C ABI) with the CPU oracle."""
import os

import numpy as np
import pytest

import oracle
from paper_2303_02471_gb300 import synth

from gpu_helpers import assert_matches_oracle, upload

pytestmark = pytest.mark.gpu

INF = (1 << 63) - 1
NCPU = len(os.sched_getaffinity(0))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(A, B, dtype=None, **cfg):
    from paper_2303_02471_gb300 import ops
    dA, dB = upload(A, dtype), upload(B, dtype)
    C, plan = ops.spgemm(dA, dB, ops.Config(**cfg) if cfg else None)
    plan.check()
    return C, plan


def test_fig1_example():
    from helpers import from_dense, read_golden
    g = read_golden("fig1.txt")
    A, B = from_dense(g["A"]), from_dense(g["B"])
    C, plan = _run(A, B)
    assert np.array_equal(plan.op_counts().cpu().numpy(), g["OP"][0].astype(np.int64))
    assert_matches_oracle(C, A, B, tau=0.0)


@pytest.mark.parametrize("t", [0, 40, None, INF])
def test_workload1_lap2d(t):
    A, B = synth.workload(1)
    C, plan = _run(A, B, t=t)
    assert_matches_oracle(C, A, B)
    assert C.nnz == 12676


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("seed", range(60))
def test_fuzz(seed, dtype):
    A, B = synth.fuzz_pair(seed, dtype=dtype)
    C, _ = _run(A, B)
    assert_matches_oracle(C, A, B)


@pytest.mark.parametrize("t", [0, 3, 20, INF])
@pytest.mark.parametrize("seed", [5, 11, 23, 42, 77])
def test_fuzz_threshold_invariance(seed, t):
    A, B = synth.fuzz_pair(seed)
    C, _ = _run(A, B, t=t)
    assert_matches_oracle(C, A, B)


@pytest.mark.parametrize("hmax", [256, 1024, 8192])
@pytest.mark.parametrize("t", [0, 40, None, INF])
def test_rmat_every_bin(t, hmax):
    """A power-law pattern with Op_j from 1 to ~10^5 crosses every bin."""
    A = synth.rmat(13, seed=2, col_cap=600)
    C, plan = _run(A, A, t=t, hash_cta_max=hmax)
    assert_matches_oracle(C, A, A, nthreads=NCPU)
    info = plan.info()
    assert info["products"] == int(oracle.op_counts(A, A).sum())


@pytest.mark.parametrize("cache", [0, 3 * 4 * 256, None])
def test_dense_flag_cache_budgets(cache):
    """Dense columns with and without flags kept from the symbolic phase
    (no cache, a cache for only the first few columns, the default)."""
    A = synth.rmat(13, seed=4, col_cap=600)
    C, plan = _run(A, A, t=0, dense_cache_bytes=cache)
    assert plan.info()["bins"][13] > 3
    assert_matches_oracle(C, A, A, nthreads=NCPU)


GROUP_OPMAX = (8, 16, 32, 64, 128, 256)  # Op_j bound of each lane-group bin


@pytest.mark.parametrize("acc", ["hash", "auto"])
@pytest.mark.parametrize("promote,pct", [(1, 125), (2, 400), (1, 300)])
def test_table_size_and_group_promotion(promote, pct, acc):
    """Larger or smaller hash tables and light columns moved up the lane-group
    bins give the oracle's C; the bin histogram follows the shifted binning
    rule (a column's smallest group bin, `promote` bins up, at most the last)."""
    A = synth.rmat(13, seed=2, col_cap=600)
    C, plan = _run(A, A, t=3000, hash_cta_max=1024, table_slots_pct=pct, group_promote=promote,
                   small_accumulator=acc)
    assert_matches_oracle(C, A, A, nthreads=NCPU)
    op = oracle.op_counts(A, A)
    want = np.zeros(6, dtype=np.int64)
    light = op[(op > 0) & (op <= 256)]
    first = np.searchsorted(np.array(GROUP_OPMAX), light)  # smallest bin with opmax >= Op_j
    np.add.at(want, np.minimum(first + promote, 5), 1)
    assert plan.info()["bins"][1:7] == want.tolist()


def test_op_counts_and_bins():
    A = synth.rmat(12, seed=5, col_cap=300)
    B = synth.random_z(A.ncols, 0, 12, seed=6)
    C, plan = _run(A, B, t=40)
    op = plan.op_counts().cpu().numpy()
    assert np.array_equal(op, oracle.op_counts(A, B))
    bins = plan.info()["bins"]
    assert bins[0] == int((op == 0).sum())
    assert bins[13] == int((op >= 40).sum())
    assert sum(bins) == A.ncols


def test_workload2_random_full():
    A, B = synth.workload(2)
    C, plan = _run(A, B)
    assert_matches_oracle(C, A, B, nthreads=NCPU)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_workload2_random_reduced(dtype):
    A = synth.random_z(1 << 16, 1, 8, seed=0, dtype=dtype)
    B = synth.random_z(1 << 16, 1, 8, seed=1, dtype=dtype)
    C, _ = _run(A, B)
    assert_matches_oracle(C, A, B)


def test_workload3_rmat_full():
    """Full-size R-MAT product (2^18, ~672M products) against the oracle."""
    A, B = synth.workload(3)
    C, plan = _run(A, B)
    assert_matches_oracle(C, A, B, nthreads=NCPU)


@pytest.mark.parametrize("t", [0, INF])
def test_workload3_threshold_extremes_pattern(t):
    """H-HASH(0) is all-SPA and H-HASH(inf) all-hash (Section 3.3); both give
    the same structure as the default split on a reduced R-MAT."""
    A = synth.rmat(15, seed=0, col_cap=2000)
    C, _ = _run(A, A, t=t)
    assert_matches_oracle(C, A, A, nthreads=NCPU)


def _tall(m, n, zlo, zhi, seed):
    """m x n with Z ~ U{zlo..zhi} distinct uniform rows per column."""
    rng = np.random.default_rng(seed)
    z = rng.integers(zlo, zhi + 1, size=n)
    rows = np.concatenate([rng.choice(m, int(k), replace=False) for k in z])
    cols = np.repeat(np.arange(n), z)
    return synth.from_coo(m, n, rows, cols, rng.standard_normal(rows.size))


@pytest.mark.parametrize("t", [0, None, INF])
def test_tall_products_flags_in_global_scratch(t):
    # m = 2^20 rows, 94 % of them holding entries (no row compaction): a
    # dense column's flags (32,768 words, 256 KB) and a CTA table's row
    # bitmap (128 KB) exceed shared memory and live in the per-CTA global
    # scratch; Op_j spans the CTA bins and the global table
    A = _tall(1 << 20, 3000, 900, 1100, seed=21)
    B = _tall(3000, 600, 1, 12, seed=22)
    C, plan = _run(A, B, t=t)
    bins = plan.info()["bins"]
    if t == 0:
        assert bins[13] == sum(bins[1:])
    if t == INF:
        assert bins[12] > 0 and sum(bins[7:12]) > 0
    assert_matches_oracle(C, A, B, nthreads=NCPU)


def test_tall_products_float32_all_dense():
    A = _tall(1 << 20, 3000, 900, 1100, seed=23).astype(np.float32)
    B = _tall(3000, 600, 1, 12, seed=24).astype(np.float32)
    C, _ = _run(A, B, dtype=np.float32, t=0)
    assert_matches_oracle(C, A, B, nthreads=NCPU)


def test_identity_is_bit_exact():
    from helpers import identity
    A = synth.random_z(5000, 1, 9, seed=5)
    I = identity(5000)
    for L, R in ((A, I), (I, A)):
        C, _ = _run(L, R)
        G = C.to_host()
        assert np.array_equal(G.colptr, A.colptr)
        assert np.array_equal(G.rowidx, A.rowidx)
        assert np.array_equal(G.values, A.values)


def test_unsorted_input_columns():
    rng = np.random.default_rng(3)
    A = synth.random_pattern(rng, 3000, 2000, 0.01, shuffle=True)
    B = synth.random_pattern(rng, 2000, 1500, 0.01, shuffle=True)
    C, _ = _run(A, B, t=40)
    assert_matches_oracle(C, A, B)


def test_repeat_numeric_is_stable():
    from paper_2303_02471_gb300 import ops
    A = synth.rmat(12, seed=9, col_cap=400)
    dA = upload(A)
    _, _, plan = ops.spgemm_symbolic(dA, dA)
    C1 = ops.spgemm_numeric(plan, dA, dA)
    C2 = ops.spgemm_numeric(plan, dA, dA)
    plan.check()
    assert (C1.rowidx == C2.rowidx).all()
    ref = oracle.spgemm(A, A)
    assert_matches_oracle(C1, A, A, ref=ref)
    assert_matches_oracle(C2, A, A, ref=ref)


@pytest.mark.parametrize("stream", ["default", "side", "graph"])
def test_numeric_forks_group_bins_and_joins(stream):
    """Dense and lane-group bins together: the group bins run on streams
    forked from the caller's and joined back before the call's later work,
    on the legacy default stream, a side stream, and inside a CUDA graph."""
    import torch
    from paper_2303_02471_gb300 import ops
    A = synth.rmat(12, seed=12, col_cap=400)
    dA = upload(A)
    _, _, plan = ops.spgemm_symbolic(dA, dA, ops.Config(t=64))
    bins = plan.info()["bins"]
    assert bins[13] > 0 and sum(bins[1:7]) > 0
    ref = oracle.spgemm(A, A)
    if stream == "default":
        C = ops.spgemm_numeric(plan, dA, dA)
        total = C.values.double().abs().sum().item()  # later work on the caller's stream
    else:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            C = ops.spgemm_numeric(plan, dA, dA)
            if stream == "graph":
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    ops.spgemm_numeric(plan, dA, dA, C.rowidx, C.values)
                C.values.zero_()
                g.replay()
            total = C.values.double().abs().sum().item()
    plan.check()
    C_ref, absC = ref
    assert abs(total - float(np.abs(C_ref.values).sum())) <= 1e-9 * float(absC.sum())
    assert_matches_oracle(C, A, A, ref=ref)


# ----------------------------------------------------------- errors
def _status(fn):
    from paper_2303_02471_gb300._native import SpgError
    with pytest.raises(SpgError) as e:
        fn()
    return e.value.name


def test_invalid_inputs_are_rejected():
    import torch
    from paper_2303_02471_gb300 import ops
    A = synth.random_z(100, 1, 5, seed=1)
    dA = upload(A)
    bad = dA.with_values(dA.values)
    bad_cp = dA.colptr.clone()
    bad_cp[10] = bad_cp[11] + 3  # not monotone
    assert _status(lambda: ops.spgemm(ops.CscMatrix(100, 100, bad_cp, dA.rowidx, dA.values), dA)) == "SPG_ERR_INVALID"
    bad_row = dA.rowidx.clone()
    bad_row[7] = 100  # out of range
    assert _status(lambda: ops.spgemm(dA, ops.CscMatrix(100, 100, dA.colptr, bad_row, dA.values))) == "SPG_ERR_INVALID"
    last = dA.colptr.clone()
    last[-1] -= 1  # colptr[n] != nnz
    assert _status(lambda: ops.spgemm(ops.CscMatrix(100, 100, last, dA.rowidx, dA.values), dA)) == "SPG_ERR_INVALID"
    # shape mismatch and dtype mismatch
    B = upload(synth.random_z(99, 1, 5, seed=2))
    assert _status(lambda: ops.spgemm(dA, B)) == "SPG_ERR_INVALID"
    assert _status(lambda: ops.spgemm(dA, dA.with_values(dA.values.float()))) == "SPG_ERR_INVALID"
    del bad, torch


def test_numeric_reports_rows_outside_the_plan():
    # the forward passes number only the rows of A that hold entries (R-MAT
    # leaves many empty); a numeric call whose A has an entry in a row that
    # was empty when the plan was made is reported, not walked
    from paper_2303_02471_gb300 import ops
    A = synth.rmat(12, seed=9, col_cap=400)
    present = np.unique(A.rowidx)
    assert present.size < 0.9 * A.nrows
    empty = int(np.setdiff1d(np.arange(A.nrows), present)[0])
    dA = upload(A)
    _, _, plan = ops.spgemm_symbolic(dA, dA)
    plan.check()
    moved = dA.rowidx.clone()
    moved[0] = empty
    ops.spgemm_numeric(plan, ops.CscMatrix(A.nrows, A.ncols, dA.colptr, moved, dA.values), dA)
    assert _status(plan.check) == "SPG_ERR_INVALID"


def test_workspace_too_small():
    import torch
    from paper_2303_02471_gb300 import _native as N
    from paper_2303_02471_gb300 import ops
    import ctypes
    A = upload(synth.random_z(500, 1, 5, seed=1))
    need = ops.workspace_size(A, A)
    ws = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    cp = torch.empty(A.ncols + 1, dtype=torch.int64, device="cuda")
    nnz, h = ctypes.c_int64(), ctypes.c_void_p()
    cA = ops._csc(A)
    rc = N.lib().spgemm_symbolic(None, ctypes.byref(cA), ctypes.byref(cA), None, ctypes.c_void_p(ws.data_ptr()),
                                 ws.numel(), ctypes.c_void_p(cp.data_ptr()), ctypes.byref(nnz),
                                 ctypes.byref(h), ops._stream())
    assert N.STATUS[rc] == "SPG_ERR_WORKSPACE"
    assert h.value is None


@pytest.mark.parametrize("t", [None, INF])
def test_table_overflow_is_reported_not_hung(t):
    A = synth.rmat(11, seed=3, col_cap=300)
    assert _status(lambda: _run(A, A, t=t, table_shrink=4)) == "SPG_ERR_TABLE_OVERFLOW"


def test_empty_shapes():
    for seed in range(6):
        A, B = synth.fuzz_pair(seed)
        C, _ = _run(A, B)
        assert_matches_oracle(C, A, B)


def test_bulk_wait_time_out_is_reported_without_a_fault():
    """The dense kernel's wait for a column's kept flags gives up at once
    (test knob): the copy it waited for still lands before the CTA exits, the
    call reports SPG_ERR_TIMEOUT, and the next product runs clean.  4096 rows
    that all hold entries give 128-word flags, which the kernel stages by a
    bulk copy."""
    from paper_2303_02471_gb300 import ops
    A = synth.random_z(4096, 30, 60, seed=21)
    assert np.unique(A.rowidx).size == A.nrows
    dA = upload(A)
    _, _, plan = ops.spgemm_symbolic(dA, dA, ops.Config(t=64, test_wait_timeout=True))
    assert plan.info()["bins"][13] == A.ncols
    ops.spgemm_numeric(plan, dA, dA)
    assert _status(plan.check) == "SPG_ERR_TIMEOUT"
    plan.destroy()
    C, plan2 = _run(A, A, t=64)
    assert_matches_oracle(C, A, A, nthreads=NCPU)


def test_handle_serves_several_plans():
    """Plans made with one handle fork onto its side streams (dense and
    lane-group bins together) and read back through its buffer; the handle
    is released after them."""
    import torch
    from paper_2303_02471_gb300 import ops
    h = ops.Handle(torch.cuda.current_device())
    A = synth.rmat(12, seed=12, col_cap=400)
    B = synth.rmat(12, seed=13, col_cap=400)
    dA, dB = upload(A), upload(B)
    plans, outs = [], []
    for X, Y in ((dA, dA), (dA, dB), (dB, dA)):
        _, _, plan = ops.spgemm_symbolic(X, Y, ops.Config(t=64), lib_handle=h)
        assert any(plan.bin_streams())
        outs.append(ops.spgemm_numeric(plan, X, Y))
        plans.append(plan)
    for plan in plans:
        plan.check()
    for (X, Y), C in zip(((A, A), (A, B), (B, A)), outs):
        assert_matches_oracle(C, X, Y)
    for plan in plans:
        plan.destroy()
    h.destroy()


def test_serial_bins_match_forked_bins():
    # side_streams = 0 runs every bin in order on the caller's stream: same C
    from paper_2303_02471_gb300 import ops
    A = synth.rmat(12, seed=14, col_cap=400)
    dA = upload(A)
    C1, p1 = ops.spgemm(dA, dA, ops.Config(t=64))
    C2, p2 = ops.spgemm(dA, dA, ops.Config(t=64, side_streams=False))
    assert any(p1.bin_streams()) and not any(p2.bin_streams())
    p1.check()
    p2.check()
    assert (C1.rowidx == C2.rowidx).all()
    ref = oracle.spgemm(A, A)
    assert_matches_oracle(C1, A, A, ref=ref)
    assert_matches_oracle(C2, A, A, ref=ref)


# ------------------------------------------------------------------- ESC
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("seed", range(40))
def test_esc_fuzz(seed, dtype):
    A, B = synth.fuzz_pair(seed, dtype=dtype)
    C, _ = _run(A, B, small_accumulator="esc")
    assert_matches_oracle(C, A, B)


@pytest.mark.parametrize("t", [None, 40, INF])
def test_esc_rmat_every_bin(t):
    # light columns by ESC beside CTA hash bins, the global table and the dense SPA
    A = synth.rmat(13, seed=2, col_cap=600)
    C, plan = _run(A, A, t=t, hash_cta_max=1024, small_accumulator="esc")
    assert sum(plan.info()["bins"][1:7]) > 0
    assert_matches_oracle(C, A, A, nthreads=NCPU)


def test_esc_workload2_random_full():
    """The random 2^20 product (every column Op_j <= 64) with the ESC accumulator."""
    A, B = synth.workload(2)
    C, plan = _run(A, B, small_accumulator="esc")
    assert sum(plan.info()["bins"][1:7]) == B.ncols - plan.info()["bins"][0]
    assert_matches_oracle(C, A, B, nthreads=NCPU)


def test_esc_tall_and_unsorted():
    # 2^20 rows (20-bit rows in the keys) and columns whose rows come unsorted
    rng = np.random.default_rng(7)
    A = _tall(1 << 20, 4000, 1, 12, seed=25)
    B = _tall(4000, 3000, 1, 9, seed=26)
    perm = np.concatenate([rng.permutation(np.arange(A.colptr[j], A.colptr[j + 1])) for j in range(A.ncols)])
    Au = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx[perm], A.values[perm])
    C, _ = _run(Au, B, small_accumulator="esc")
    assert_matches_oracle(C, A, B, nthreads=NCPU)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_esc_sort_forms(dtype):
    # 2^21 rows, 15/16 of them holding entries (no row compaction: 21-bit rows
    # in the keys).  Composite keys of (column place, row, position) fit 32
    # bits in the bins of Op_j <= 32 and <= 64 (the count over a window) but
    # not in those of <= 8 and <= 16 (the count over the column alone); the
    # bins of <= 128 and <= 256 keep the radix sort.
    rng = np.random.default_rng(31)
    m, k = 1 << 21, 1 << 18
    arow = rng.permutation(m).reshape(k, 8)
    arow[1::2, 0] = arow[0::2, 0]  # A's columns 2q and 2q + 1 share a row
    A = synth.from_coo(m, k, arow.ravel(), np.repeat(np.arange(k), 8), rng.standard_normal(m))
    n = 6000
    z = rng.integers(1, 9, size=n)  # Op_j = 8 z: the bins of <= 8 .. <= 64
    z[:60] = rng.integers(9, 33, size=60)  # Op_j of 72..256
    cols = []
    for j in range(n):
        r = 2 * rng.choice(k // 2, int(z[j]), replace=False) + rng.integers(0, 2, int(z[j]))
        if j % 3 == 0 and z[j] >= 2:
            r[1] = r[0] ^ 1  # both columns of a pair: C rows met twice
        cols.append(r)
    B = synth.from_coo(k, n, np.concatenate(cols), np.repeat(np.arange(n), z), rng.standard_normal(int(z.sum())))
    C, plan = _run(A, B, dtype=dtype, small_accumulator="esc")
    bins = plan.info()["bins"]
    assert all(bins[b] > 0 for b in range(1, 7)), bins
    assert C.rowidx.numel() < int(plan.op_counts().sum())  # equal keys were merged
    assert_matches_oracle(C, A, B, nthreads=NCPU)


def test_esc_sums_do_not_depend_on_timing():
    # every column light (Op_j <= 225): the whole C comes from ESC, whose sums
    # run in sorted order, so two calls agree bit for bit
    from paper_2303_02471_gb300 import ops
    A = synth.random_z(20000, 1, 15, seed=8)
    B = synth.random_z(20000, 1, 15, seed=9)
    dA, dB = upload(A), upload(B)
    _, _, plan = ops.spgemm_symbolic(dA, dB, ops.Config(small_accumulator="esc"))
    assert sum(plan.info()["bins"][7:]) == 0
    C1 = ops.spgemm_numeric(plan, dA, dB)
    v1 = C1.values.clone()
    C2 = ops.spgemm_numeric(plan, dA, dB)
    plan.check()
    assert (C2.values == v1).all()
    assert_matches_oracle(C2, A, B)


# ----------------------------------------------------------- single pass
def _single(A, B, dtype=None, **cfg):
    from paper_2303_02471_gb300 import ops
    dA, dB = upload(A, dtype), upload(B, dtype)
    C, plan = ops.spgemm_single_pass(dA, dB, ops.Config(**cfg) if cfg else None)
    plan.check()
    return C, plan


@pytest.mark.parametrize("acc", ["hash", "esc"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("seed", range(20))
def test_single_pass_fuzz(seed, dtype, acc):
    A, B = synth.fuzz_pair(seed, dtype=dtype)
    C, _ = _single(A, B, small_accumulator=acc)
    assert_matches_oracle(C, A, B)


@pytest.mark.parametrize("acc", ["hash", "esc"])
@pytest.mark.parametrize("t", [0, 40, None, INF])
def test_single_pass_rmat_every_bin(t, acc):
    # every accumulator writing to Op_j-sized slots: lane groups or ESC, CTA
    # tables, the global table and the dense SPA (flags set by a first walk)
    A = synth.rmat(13, seed=2, col_cap=600)
    C, plan = _single(A, A, t=t, hash_cta_max=1024, small_accumulator=acc)
    assert_matches_oracle(C, A, A, nthreads=NCPU)


@pytest.mark.parametrize("acc", ["hash", "esc"])
def test_single_pass_workload2_random_full(acc):
    A, B = synth.workload(2)
    C, _ = _single(A, B, small_accumulator=acc)
    assert_matches_oracle(C, A, B, nthreads=NCPU)


def test_single_pass_workload1_and_tall():
    A, B = synth.workload(1)
    C, _ = _single(A, B, t=12)
    assert_matches_oracle(C, A, B)
    assert C.nnz == 12676
    A = _tall(1 << 20, 3000, 900, 1100, seed=21)
    B = _tall(3000, 600, 1, 12, seed=22)
    for t in (0, INF):
        C, _ = _single(A, B, t=t)
        assert_matches_oracle(C, A, B, nthreads=NCPU)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("t", [0, INF])
def test_single_pass_long_columns_and_empty_runs(t, dtype):
    """The copy into C spreads a column over as many tiles of C's positions
    as it spans and skips runs of empty columns: a few columns of tens of
    thousands of entries among runs of empty and one-entry columns."""
    rng = np.random.default_rng(41)
    A = _tall(60000, 64, 400, 800, seed=40)
    n = 700
    z = np.zeros(n, dtype=np.int64)
    z[rng.choice(n, 150, replace=False)] = 1   # one-entry columns
    z[[3, 350, 351, 699]] = 64                  # long columns of C
    rows = np.concatenate([rng.choice(64, int(k), replace=False) for k in z])
    cols = np.repeat(np.arange(n), z)
    B = synth.from_coo(64, n, rows, cols, rng.standard_normal(rows.size))
    A, B = A.with_values(A.values.astype(dtype)), B.with_values(B.values.astype(dtype))
    C, _ = _single(A, B, t=t)
    assert C.nnz > 4 * 40000
    assert_matches_oracle(C, A, B, nthreads=NCPU)


def test_single_pass_plan_serves_numeric_and_backward():
    import torch
    from paper_2303_02471_gb300 import ops
    A = synth.rmat(12, seed=9, col_cap=400)
    dA = upload(A)
    C1, plan = ops.spgemm_single_pass(dA, dA, ops.Config(t=64))
    C2 = ops.spgemm_numeric(plan, dA, dA)
    plan.check()
    assert (C1.rowidx == C2.rowidx).all()
    ref = oracle.spgemm(A, A)
    assert_matches_oracle(C2, A, A, ref=ref)
    dc = torch.ones(C1.nnz, dtype=torch.float64, device="cuda")
    gA, gB = ops.spgemm_backward(plan, dA, dA, C1, dc)
    plan.check()
    rA, rB = oracle.backward(A, A, C1.to_host(), np.ones(C1.nnz))
    Aa = A.with_values(np.abs(A.values))
    sA, sB = oracle.backward(Aa, Aa, C1.to_host(), np.ones(C1.nnz))
    assert np.all(np.abs(gA.cpu().numpy() - rA) <= 1e-12 * sA)
    assert np.all(np.abs(gB.cpu().numpy() - rB) <= 1e-12 * sB)


def test_single_pass_workspace_too_small():
    import ctypes
    import torch
    from paper_2303_02471_gb300 import _native as N
    from paper_2303_02471_gb300 import ops
    A = upload(synth.random_z(800, 1, 6, seed=4))
    need = ops.single_pass_workspace_size(A, A)
    assert need > ops.workspace_size(A, A, ops.Config(dense_cache_bytes=0))
    ws = torch.empty(need - 4096, dtype=torch.uint8, device="cuda")
    cp = torch.empty(A.ncols + 1, dtype=torch.int64, device="cuda")
    nnz, h = ctypes.c_int64(), ctypes.c_void_p()
    cA = ops._csc(A)
    rc = N.lib().spgemm_single_pass(ops.handle().ptr, ctypes.byref(cA), ctypes.byref(cA), None,
                                    ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(cp.data_ptr()),
                                    ctypes.byref(nnz), ctypes.byref(h), ops._stream())
    assert N.STATUS[rc] == "SPG_ERR_WORKSPACE" and h.value is None


# ------------------------------------------------ hash tables in both phases
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("seed", range(30))
def test_hash_fuzz(seed, dtype):
    A, B = synth.fuzz_pair(seed, dtype=dtype)
    C, _ = _run(A, B, small_accumulator="hash")
    assert_matches_oracle(C, A, B)


@pytest.mark.parametrize("t", [None, 40, INF])
def test_hash_rmat_every_bin(t):
    A = synth.rmat(13, seed=2, col_cap=600)
    C, plan = _run(A, A, t=t, hash_cta_max=1024, small_accumulator="hash")
    assert sum(plan.info()["bins"][1:7]) > 0
    assert_matches_oracle(C, A, A, nthreads=NCPU)


def test_hash_workload2_random_full():
    A, B = synth.workload(2)
    C, _ = _run(A, B, small_accumulator="hash")
    assert_matches_oracle(C, A, B, nthreads=NCPU)

"""The row-wise (CSR) form and column sharding, through the CUDA path.

CSR: C = A B with A, B and C in CSR, against the oracle's C moved to CSR by
the oracle's transpose (the CSR arrays of M are the CSC arrays of M^T).
Sharding: the column blocks of B that shard.column_ranges deals to 2, 4 and
8 ranks, each multiplied on the GPU, concatenate to the oracle's C."""
import os

import numpy as np
import pytest

import oracle
from paper_2303_02471_gb300 import shard, synth

from gpu_helpers import TAU, upload

pytestmark = pytest.mark.gpu

NCPU = len(os.sched_getaffinity(0))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _csr_dev(M, dtype):
    """Device CSR of a host CSC matrix M (arrays of M^T), and the order of
    its entries in M's CSC storage."""
    from paper_2303_02471_gb300 import ops
    T, perm = oracle.transpose(M)
    vals = np.asarray(M.values)[perm].astype(dtype)
    return ops.CsrMatrix.from_host(M.nrows, M.ncols, T.colptr, T.rowidx, vals), perm


def _within(got, want, scale, tau, what):
    err = np.abs(np.asarray(got, dtype=np.float64) - want)
    bad = err > tau * scale
    assert not bad.any(), f"{what}: {int(bad.sum())} entries off"


def _check_csr(A, B, dtype, seed=0, **cfg):
    import torch
    from paper_2303_02471_gb300 import ops
    dA, pA = _csr_dev(A, dtype)
    dB, pB = _csr_dev(B, dtype)
    C, plan = ops.spgemm_csr(dA, dB, ops.Config(**cfg) if cfg else None)
    plan.check()
    ref, absref = oracle.spgemm(A, B, nthreads=NCPU)
    R, pC = oracle.transpose(ref)  # C in CSR: R.colptr = row pointers, R.rowidx = column indices
    tau = TAU[np.dtype(dtype)]
    assert np.array_equal(C.rowptr.cpu().numpy(), R.colptr)
    assert np.array_equal(C.colidx.cpu().numpy(), R.rowidx)
    _within(C.values.cpu().numpy(), R.values, absref[pC], tau, "C")
    # backward: dC on pattern(C) in CSR order, the oracle's gradients in CSC order
    rng = np.random.default_rng(seed)
    dc = rng.standard_normal(C.nnz).astype(dtype)
    gA, gB = ops.spgemm_csr_backward(plan, dA, dB, C, torch.as_tensor(dc, device="cuda"))
    plan.check()
    dc_csc = np.empty(C.nnz)
    dc_csc[pC] = dc
    rA, rB = oracle.backward(A, B, ref, dc_csc)
    sA, sB = oracle.backward(A.with_values(np.abs(A.values)), B.with_values(np.abs(B.values)), ref, np.abs(dc_csc))
    _within(gA.cpu().numpy(), rA[pA], sA[pA], tau, "dA")
    _within(gB.cpu().numpy(), rB[pB], sB[pB], tau, "dB")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("seed", range(12))
def test_csr_fuzz(seed, dtype):
    A, B = synth.fuzz_pair(seed, dtype=dtype)
    _check_csr(A, B, dtype, seed)


@pytest.mark.parametrize("t", [0, None, (1 << 63) - 1])
def test_csr_rmat(t):
    A = synth.rmat(12, seed=4, col_cap=400)
    B = synth.rmat(12, seed=5, col_cap=400)
    _check_csr(A, B, np.float64, 1, t=t)


@pytest.fixture(scope="module")
def rmat18():
    A, _ = synth.workload(3)
    return A, oracle.spgemm(A, A, nthreads=NCPU), oracle.op_counts(A, A)


@pytest.mark.parametrize("world", [2, 4, 8])
def test_column_shards_of_rmat18_concatenate_to_the_product(rmat18, world):
    """R-MAT 2^18 (C = A A): every rank's column block of B multiplied on the
    GPU; the blocks side by side are the oracle's C (structure bit-exact,
    values within 1e-12 of the sums of |terms|), and the blocks carry about
    equal shares of the products."""
    from paper_2303_02471_gb300 import ops
    A, (ref, absref), op = rmat18
    dA = upload(A)
    blocks, loads = [], []
    for s, e in shard.column_ranges(op, world):
        Bb = shard.column_block(A, s, e)
        C, plan = ops.spgemm(dA, upload(Bb))
        plan.check()
        loads.append(plan.info()["products"])
        blocks.append(C.to_host())
        del C, plan
    assert sum(loads) == int(op.sum())
    assert max(loads) - min(loads) <= 2 * int(op.max())
    full = shard.concat_columns(blocks)
    assert np.array_equal(full.colptr, ref.colptr)
    assert np.array_equal(full.rowidx, ref.rowidx)
    _within(full.values, ref.values, absref, 1e-12, "C")

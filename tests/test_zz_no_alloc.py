"""The transpose entry point that allocates nothing (for callers that cannot
call cudaMalloc or pass a workspace), checked against spg_csc_transpose on
two calls in a row.  Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

from paper_2303_02471_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _noalloc(M):
    import torch
    from paper_2303_02471_gb300 import _native as N
    from paper_2303_02471_gb300 import ops
    cp = torch.empty(M.nrows + 1, dtype=torch.int64, device="cuda")
    row = torch.empty(M.nnz, dtype=torch.int32, device="cuda")
    val = torch.empty(M.nnz, dtype=M.dtype, device="cuda")
    perm = torch.empty(M.nnz, dtype=torch.int64, device="cuda")
    st = N.lib().spg_csc_transpose_noalloc(ctypes.byref(ops._csc(M)), ops._ptr(cp), ops._ptr(row), ops._ptr(val),
                                            ops._ptr(perm), ops._stream())
    return st, cp, row, val, perm


def test_noalloc_transpose_matches_workspace_transpose_twice():
    import torch
    from paper_2303_02471_gb300 import ops
    from gpu_helpers import upload
    rng = np.random.default_rng(2)
    mats = [synth.rmat(12, seed=1, col_cap=300), synth.random_pattern(rng, 4, 5000, 1.0, dtype=np.float32)]
    for M in mats:  # two calls in a row, the second reusing the shared scratch
        dM = upload(M)
        T, perm = ops.csc_transpose(dM)
        st, cp, row, val, pm = _noalloc(dM)
        torch.cuda.synchronize()
        assert st == 0
        assert torch.equal(cp, T.colptr)
        assert torch.equal(row, T.rowidx)
        assert torch.allclose(val, T.values, rtol=0, atol=0)
        assert torch.equal(pm, perm)


def test_noalloc_transpose_rejects_beyond_limit():
    import torch
    from paper_2303_02471_gb300 import _native as N
    from paper_2303_02471_gb300 import ops
    # 3 million entries need more than the 32 MiB of scratch; rejected before
    # any device work (the arrays are never touched)
    dummy = torch.empty(1, dtype=torch.int64, device="cuda")
    M = N.SpgCsc(1000, 1000, 3_000_000, dummy.data_ptr(), dummy.data_ptr(), None, 0)
    st = N.lib().spg_csc_transpose_noalloc(ctypes.byref(M), ops._ptr(dummy), ops._ptr(dummy), None, None,
                                            ops._stream())
    assert N.STATUS[st] == "SPG_ERR_WORKSPACE"

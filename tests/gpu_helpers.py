"""Helpers for the GPU parity tests: upload, run through the C ABI, compare."""
import numpy as np

import oracle

TAU = {np.dtype(np.float64): 1e-12, np.dtype(np.float32): 1e-5}


def upload(M, dtype=None):
    import torch
    from paper_2303_02471_gb300.ops import CscMatrix
    tdt = {None: None, np.float64: torch.float64, np.float32: torch.float32}[dtype]
    return CscMatrix.from_host(M, device="cuda", dtype=tdt)


def assert_matches_oracle(C_gpu, A_host, B_host, nthreads=1, tau=None, ref=None):
    """Structure bit-exact; |c - c_ref| <= tau * sum|a b| per entry (exact when
    the sum is 0).  Returns the oracle result."""
    C, absC = ref if ref is not None else oracle.spgemm(A_host, B_host, nthreads=nthreads)
    G = C_gpu.to_host()
    vdt = np.dtype(G.values.dtype)
    tau = TAU[vdt] if tau is None else tau
    assert G.nrows == C.nrows and G.ncols == C.ncols
    assert np.array_equal(G.colptr, C.colptr), "column pointers differ"
    assert np.array_equal(G.rowidx, C.rowidx), "row indices differ"
    got = G.values.astype(np.float64)
    err = np.abs(got - C.values)
    bound = tau * absC
    bad = err > bound
    if bad.any():
        i = int(np.argmax(err - bound))
        raise AssertionError(f"{int(bad.sum())} values out of tolerance; worst at {i}: "
                             f"got {got[i]!r} want {C.values[i]!r} bound {bound[i]!r}")
    return C, absC

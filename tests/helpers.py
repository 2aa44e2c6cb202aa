"""Test-side helpers: dense conversions, golden fixtures, comparisons."""
import os

import numpy as np

from paper_2303_02471_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def to_dense(M) -> np.ndarray:
    D = np.zeros((M.nrows, M.ncols), dtype=np.float64)
    for j in range(M.ncols):
        lo, hi = int(M.colptr[j]), int(M.colptr[j + 1])
        np.add.at(D[:, j], M.rowidx[lo:hi].astype(np.int64),
                  np.asarray(M.values[lo:hi], dtype=np.float64))
    return D


def to_pattern(M) -> np.ndarray:
    P = np.zeros((M.nrows, M.ncols), dtype=np.int64)
    for j in range(M.ncols):
        lo, hi = int(M.colptr[j]), int(M.colptr[j + 1])
        P[M.rowidx[lo:hi], j] = 1
    return P


def from_dense(D: np.ndarray) -> synth.CSC:
    cols, rows = np.nonzero(D.T)
    return synth.from_coo(D.shape[0], D.shape[1], rows, cols, D[rows, cols])


def read_golden(name: str) -> dict:
    """Sections of a golden text file: a header word, then rows of numbers."""
    out, key = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line[0].isalpha():
                key = line
                out[key] = []
            else:
                out[key].append([float(v) for v in line.split()])
    return {k: np.array(v) for k, v in out.items()}


def identity(n: int) -> synth.CSC:
    return synth.CSC(n, n, np.arange(n + 1, dtype=np.int64),
                     np.arange(n, dtype=np.int32), np.ones(n))


def scipy_csc(M):
    import scipy.sparse as sp
    return sp.csc_matrix((np.asarray(M.values, dtype=np.float64),
                          M.rowidx.astype(np.int64), M.colptr),
                         shape=(M.nrows, M.ncols))


def transpose(M):
    """CSC of M^T with rows sorted, and perm: values_T = M.values[perm]."""
    n_e = int(M.colptr[-1])
    cols = np.repeat(np.arange(M.ncols), np.diff(M.colptr))
    rows = M.rowidx.astype(np.int64)
    perm = np.lexsort((cols, rows))
    counts = np.bincount(rows, minlength=M.nrows).astype(np.int64)
    cp = np.zeros(M.nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=cp[1:])
    T = synth.CSC(M.ncols, M.nrows, cp, cols[perm].astype(np.int32),
                  np.asarray(M.values)[perm])
    assert T.rowidx.shape[0] == n_e
    return T, perm

"""Host logic of bench.py (no GPU): the contract's defaults, the seeded column
sample the CPU baseline times, and the gate on the recorded DRAM traffic."""
import argparse
import sys

import numpy as np
import pytest

import bench  # the repository root is on sys.path (conftest)
from paper_2303_02471_gb300 import synth


def _args(**kw):
    a = argparse.Namespace(t=None, cta_threads=None, dense_cache=None, workload=3, rmat_scale=18)
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def test_defaults_keep_the_contract(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "ours" and a.workload == 3
    assert a.warmup >= 3 and a.steps >= 1
    # the L2 flush buffer is larger than GB300's 129 MB L2
    assert bench.L2_FLUSH_BYTES > 129 * 10 ** 6


def test_column_sample_keeps_whole_columns():
    B = synth.random_z(500, 1, 9, seed=3)
    full, cols = bench.column_sample(B, 1.0, seed=0)
    assert np.array_equal(cols, np.arange(B.ncols))
    assert np.array_equal(full.colptr, B.colptr) and np.array_equal(full.rowidx, B.rowidx)
    part, cols = bench.column_sample(B, 0.3, seed=1)
    assert 0 < len(cols) < B.ncols and part.ncols == len(cols)
    for i, j in enumerate(cols):
        lo, hi = B.colptr[j], B.colptr[j + 1]
        assert np.array_equal(part.rowidx[part.colptr[i]:part.colptr[i + 1]], B.rowidx[lo:hi])
        assert np.array_equal(part.values[part.colptr[i]:part.colptr[i + 1]], B.values[lo:hi])
    again, cols2 = bench.column_sample(B, 0.3, seed=1)
    assert np.array_equal(cols, cols2)


def test_traffic_is_reported_only_for_the_captured_kernel_and_case(monkeypatch):
    t = bench.MEASURED_TRAFFIC
    got = bench.measured_traffic(t["bin"], _args())
    assert got == int(t["bytes"])  # the committed sources are the captured ones
    assert bench.measured_traffic(t["bin"] - 1, _args()) is None
    assert bench.measured_traffic(t["bin"], _args(rmat_scale=17)) is None
    assert bench.measured_traffic(t["bin"], _args(t=100)) is None
    assert bench.measured_traffic(t["bin"], _args(cta_threads=256)) is None
    assert bench.measured_traffic(t["bin"], _args(workload=2)) is None
    changed = dict(t, sources_sha256_16="0" * 16)
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", changed)
    assert bench.measured_traffic(t["bin"], _args()) is None


@pytest.mark.parametrize("k", [1, 2, 3])
def test_workload_names_match_sizes(k):
    name = bench.workload_name(_args(workload=k))
    assert isinstance(name, str) and name


def test_roofline_kernel_is_the_bin_with_most_bytes():
    nb = 14
    st = {k: [0] * nb for k in ("count", "nnz_b", "products", "nnz")}
    # a lane-group bin and the dense bin: the dense one moves more bytes
    st["count"][6], st["nnz_b"][6], st["products"][6], st["nnz"][6] = 12742, 60000, 2060514, 2053110
    st["count"][13], st["nnz_b"][13], st["products"][13], st["nnz"][13] = 90338, 1500000, 669840362, 387843925
    assert bench.dominant_bin(st, 8) == 13
    st["count"][13] = st["nnz_b"][13] = st["products"][13] = st["nnz"][13] = 0
    assert bench.dominant_bin(st, 8) == 6
    # the empty-column bin never counts
    st["count"][0] = 10 ** 6
    assert bench.dominant_bin(st, 8) == 6

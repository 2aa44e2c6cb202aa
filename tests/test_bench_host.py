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


def _sources_hash(files):
    import hashlib
    import os
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(bench.ROOT, "paper_2303_02471_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def test_traffic_is_reported_only_for_the_captured_kernel_and_case(monkeypatch):
    files = ("kernels.cuh", "numeric.cu")
    rec = {"workload": 3, "bin": 13, "capture": "c", "accumulators": (None,), "bytes": 4.0e9,
           "algorithmic_bytes": 5.0e9, "sources": files, "sources_sha256_16": _sources_hash(files)}
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", (rec,))
    got, src = bench.measured_traffic(13, 10.0e9, _args())
    assert got == 8 * 10 ** 9 and "scaled" in src  # scaled by the algorithmic bytes
    assert bench.measured_traffic(12, 10.0e9, _args())[0] is None
    assert bench.measured_traffic(13, 10.0e9, _args(t=100))[0] is None
    assert bench.measured_traffic(13, 10.0e9, _args(cta_threads=256))[0] is None
    assert bench.measured_traffic(13, 10.0e9, _args(workload=2))[0] is None
    assert bench.measured_traffic(13, 10.0e9, _args(accumulator="hash"))[0] is None
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", (dict(rec, sources_sha256_16="0" * 16),))
    assert bench.measured_traffic(13, 10.0e9, _args())[0] is None
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", None)
    assert bench.measured_traffic(13, 10.0e9, _args())[0] is None


def test_traffic_of_a_side_workload_by_its_accumulator(monkeypatch):
    files = ("esc.cu",)
    rec = {"workload": 2, "bin": 3, "capture": "c", "accumulators": (None, "esc"), "bytes": 3.0e8,
           "algorithmic_bytes": 3.0e8, "sources": files, "sources_sha256_16": _sources_hash(files)}
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", (rec,))
    assert bench.measured_traffic(3, 3.0e8, None, workload=2)[0] == 3 * 10 ** 8
    assert bench.measured_traffic(3, 3.0e8, None, workload=2, accumulator="esc")[0] == 3 * 10 ** 8
    assert bench.measured_traffic(3, 3.0e8, None, workload=2, accumulator="hash")[0] is None
    assert bench.measured_traffic(3, 3.0e8, None, workload=3)[0] is None
    assert bench.measured_traffic(3, 3.0e8, _args(workload=2))[0] == 3 * 10 ** 8


def test_backward_bytes_count_each_array_once():
    A = synth.random_z(50, 2, 2, seed=1)
    B = synth.random_z(50, 3, 3, seed=2)
    full = bench.backward_bytes(A, B, 300, 280, 8)
    no_da = bench.backward_bytes(A, B, 300, 280, 8, need_dA=False)
    assert full - no_da == 100 * 8  # dA: nnz(A) values written once


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


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_are_summarised(tmp_path):
    # nvidia-smi --format=csv,noheader,nounits rows: index, clocks.sm,
    # clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    p = tmp_path / "clocks.csv"
    p.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, [N/A], 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "a short line\n")
    s = bench.ClockSampler()
    s.proc, s.path = _DoneProc(), str(p)
    out = s.stop()
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2070.0  # median of the three numeric samples
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert not p.exists()


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler()
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

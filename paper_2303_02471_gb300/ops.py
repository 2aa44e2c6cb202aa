"""Torch-facing calls of the GB300 SpGEMM (argument marshalling only).

Torch provides device memory and the current CUDA stream; every step of the
product runs in the kernels of libspgemm.so behind the C ABI of
``include/spgemm.h``.  The names follow the ABI: :func:`spgemm_symbolic`,
:func:`spgemm_numeric`, :func:`spgemm_backward`, plus :func:`spgemm` (both
phases) and :func:`csc_transpose`.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, replace
from typing import Optional

import torch

from . import _native as N


@dataclass
class CscMatrix:
    """A CSC matrix in device memory (Section 2.1 of arXiv 2303.02471)."""

    nrows: int
    ncols: int
    colptr: torch.Tensor            # int64 [ncols + 1]
    rowidx: torch.Tensor            # int32 [nnz]
    values: Optional[torch.Tensor]  # float64 / float32 [nnz] or None

    @property
    def nnz(self) -> int:
        return int(self.rowidx.shape[0])

    @property
    def dtype(self):
        return self.values.dtype if self.values is not None else torch.float64

    @property
    def device(self):
        return self.colptr.device

    @staticmethod
    def from_host(M, device="cuda", dtype=None) -> "CscMatrix":
        """From any host object with nrows/ncols/colptr/rowidx/values (numpy)."""
        vals = torch.as_tensor(M.values)
        if dtype is not None:
            vals = vals.to(dtype)
        return CscMatrix(int(M.nrows), int(M.ncols),
                         torch.as_tensor(M.colptr, dtype=torch.int64).to(device),
                         torch.as_tensor(M.rowidx, dtype=torch.int32).to(device),
                         vals.to(device))

    def to_host(self):
        from types import SimpleNamespace
        return SimpleNamespace(nrows=self.nrows, ncols=self.ncols,
                               colptr=self.colptr.cpu().numpy(),
                               rowidx=self.rowidx.cpu().numpy(),
                               values=None if self.values is None else self.values.detach().cpu().numpy())

    def with_values(self, values: torch.Tensor) -> "CscMatrix":
        return replace(self, values=values)

    def to_torch_sparse(self) -> torch.Tensor:
        return torch.sparse_csc_tensor(self.colptr, self.rowidx.to(torch.int64), self.values,
                                       size=(self.nrows, self.ncols))

    @staticmethod
    def from_torch_sparse(T: torch.Tensor) -> "CscMatrix":
        T = T.to_sparse_csc()
        return CscMatrix(T.shape[0], T.shape[1], T.ccol_indices().to(torch.int64),
                         T.row_indices().to(torch.int32), T.values())


@dataclass
class CsrMatrix:
    """A CSR matrix in device memory (the row-wise form of Section 2.1)."""

    nrows: int
    ncols: int
    rowptr: torch.Tensor            # int64 [nrows + 1]
    colidx: torch.Tensor            # int32 [nnz]
    values: Optional[torch.Tensor]  # float64 / float32 [nnz] or None

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    @property
    def dtype(self):
        return self.values.dtype if self.values is not None else torch.float64

    @property
    def device(self):
        return self.rowptr.device

    @staticmethod
    def from_host(nrows, ncols, rowptr, colidx, values, device="cuda") -> "CsrMatrix":
        return CsrMatrix(int(nrows), int(ncols), torch.as_tensor(rowptr, dtype=torch.int64).to(device),
                         torch.as_tensor(colidx, dtype=torch.int32).to(device),
                         torch.as_tensor(values).to(device))


@dataclass
class Config:
    """Mirror of spg_config; None fields keep the library defaults."""

    t: Optional[int] = None            # H-HASH(t) threshold; N.INT64_MAX = infinity
    hash_cta_max: Optional[int] = None
    cta_threads: Optional[int] = None
    validate: Optional[bool] = None
    table_shrink: Optional[int] = None
    scratch_cap_bytes: Optional[int] = None
    dense_cache_bytes: Optional[int] = None
    side_streams: Optional[bool] = None
    test_wait_timeout: Optional[bool] = None
    small_accumulator: Optional[str] = None  # "hash", "esc" or "auto"
    table_slots_pct: Optional[int] = None    # hash-table slots per output entry, per cent (125..400)
    group_promote: Optional[int] = None      # lane-group bins a light column moves up (0..2)

    def native(self) -> N.SpgConfig:
        c = N.SpgConfig()
        N.check(N.lib().spg_config_default(ctypes.byref(c)), "spg_config_default")
        for f in ("t", "hash_cta_max", "cta_threads", "table_shrink", "scratch_cap_bytes",
                  "dense_cache_bytes", "table_slots_pct", "group_promote"):
            v = getattr(self, f)
            if v is not None:
                setattr(c, f, int(v))
        for f in ("validate", "side_streams", "test_wait_timeout"):
            v = getattr(self, f)
            if v is not None:
                setattr(c, f, int(bool(v)))
        if self.small_accumulator is not None:
            c.small_accumulator = {"hash": N.SPG_ACC_HASH, "esc": N.SPG_ACC_ESC,
                                   "auto": N.SPG_ACC_AUTO}[self.small_accumulator]
        return c


_DT = {torch.float64: N.SPG_F64, torch.float32: N.SPG_F32}


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else None


def _csc(M: CscMatrix, dtype=None) -> N.SpgCsc:
    dt = dtype if dtype is not None else M.dtype
    if dt not in _DT:
        raise TypeError(f"unsupported dtype {dt}")
    for t, want in ((M.colptr, torch.int64), (M.rowidx, torch.int32)):
        if t.dtype != want or not t.is_contiguous() or not t.is_cuda:
            raise TypeError("CSC index arrays must be contiguous CUDA int64 colptr / int32 rowidx")
    if M.values is not None and (not M.values.is_contiguous() or not M.values.is_cuda):
        raise TypeError("CSC values must be a contiguous CUDA tensor")
    return N.SpgCsc(M.nrows, M.ncols, M.nnz, M.colptr.data_ptr(), _ptr(M.rowidx),
                    _ptr(M.values), _DT[dt])


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Handle:
    """An spg_handle of one device: the side streams, events and pinned
    read-back buffer that the calls made with it use (created at once)."""

    def __init__(self, device: int):
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            N.check(N.lib().spg_create(ctypes.byref(h)), "spg_create")
        self._h = h
        self.device = device

    @property
    def ptr(self):
        if self._h is None:
            raise RuntimeError("handle destroyed")
        return self._h

    def destroy(self) -> None:
        if self._h is not None:
            N.lib().spg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


_HANDLES = {}


def handle(device=None) -> Handle:
    """The shared handle of a CUDA device (default: the current one), created
    on first use.  Calls made with one handle run their side-stream bins in
    order; give concurrent products on different streams a Handle each."""
    if device is None:
        idx = torch.cuda.current_device()
    else:
        d = torch.device(device)
        idx = d.index if d.index is not None else torch.cuda.current_device()
    h = _HANDLES.get(idx)
    if h is None:
        h = _HANDLES[idx] = Handle(idx)
    return h


class Plan:
    """Host plan of one product plus the device workspace that holds its state."""

    def __init__(self, handle: ctypes.c_void_p, workspace: torch.Tensor, A: CscMatrix,
                 B: CscMatrix, colptr: torch.Tensor, nnz: int, config: Config, lib_handle=None):
        self._h = handle
        self._lib_handle = lib_handle  # kept alive while the plan is
        self.workspace = workspace
        self.shape = (A.nrows, B.ncols)
        self.dtype = A.dtype
        self.colptr = colptr
        self.nnz = nnz
        self.config = config

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def info(self):
        nb = ctypes.c_int32()
        counts = (ctypes.c_int64 * 64)()
        prod = ctypes.c_int64()
        t = ctypes.c_int64()
        N.check(N.lib().spg_plan_info(self.handle, ctypes.byref(nb), counts, ctypes.byref(prod),
                                      ctypes.byref(t)), "spg_plan_info")
        return {"bins": list(counts[:nb.value]), "products": prod.value, "t": t.value}

    def bin_stats(self):
        arrs = [(ctypes.c_int64 * 64)() for _ in range(5)]
        N.check(N.lib().spg_plan_bin_stats(self.handle, *arrs), "spg_plan_bin_stats")
        nb = len(self.info()["bins"])
        keys = ("products", "nnz", "max_op", "max_nnz", "nnz_b")
        return {k: list(a[:nb]) for k, a in zip(keys, arrs)}

    def launch_count(self):
        s, n, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        N.check(N.lib().spg_plan_launch_count(self.handle, ctypes.byref(s), ctypes.byref(n),
                                              ctypes.byref(b)), "spg_plan_launch_count")
        return {"symbolic": s.value, "numeric": n.value, "backward": b.value}

    def bin_streams(self):
        """Per bin: True when its numeric kernel runs on a side stream."""
        side = (ctypes.c_int32 * 64)()
        N.check(N.lib().spg_plan_bin_streams(self.handle, side), "spg_plan_bin_streams")
        return [bool(x) for x in side[:len(self.info()["bins"])]]

    def set_timing(self, enable: bool = True) -> None:
        N.check(N.lib().spg_plan_set_timing(self.handle, int(bool(enable))), "spg_plan_set_timing")

    def bin_times(self):
        ms = (ctypes.c_float * 64)()
        N.check(N.lib().spg_plan_bin_times(self.handle, ms), "spg_plan_bin_times")
        return list(ms[:len(self.info()["bins"])])

    def op_counts(self) -> torch.Tensor:
        out = torch.empty(self.shape[1], dtype=torch.int64, device=self.workspace.device)
        N.check(N.lib().spg_plan_op_counts(self.handle, _ptr(out), _stream()), "spg_plan_op_counts")
        return out

    def check(self) -> None:
        N.check(N.lib().spg_plan_check(self.handle, _stream()), "spg_plan_check")

    def destroy(self) -> None:
        if self._h is not None:
            N.lib().spg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def workspace_size(A: CscMatrix, B: CscMatrix, config: Optional[Config] = None) -> int:
    cfg = (config or Config()).native()
    nbytes = ctypes.c_size_t()
    N.check(N.lib().spgemm_workspace_size(ctypes.byref(_csc(A)), ctypes.byref(_csc(B, A.dtype)),
                                          ctypes.byref(cfg), ctypes.byref(nbytes)),
            "spgemm_workspace_size")
    return nbytes.value


def spgemm_symbolic(A: CscMatrix, B: CscMatrix, config: Optional[Config] = None,
                    workspace: Optional[torch.Tensor] = None, lib_handle: Optional[Handle] = None):
    """Column pointers of C = A B, nnz(C) and the plan (synchronises).
    lib_handle: the Handle to use (default: the device's shared one)."""
    config = config or Config()
    hd = lib_handle if lib_handle is not None else handle(A.device)
    cfg = config.native()
    cA, cB = _csc(A), _csc(B, A.dtype)
    need = workspace_size(A, B, config)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=A.device)
    colptr = torch.empty(B.ncols + 1, dtype=torch.int64, device=A.device)
    nnz = ctypes.c_int64()
    h = ctypes.c_void_p()
    N.check(N.lib().spgemm_symbolic(hd.ptr, ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(cfg),
                                    _ptr(workspace), workspace.numel(), _ptr(colptr),
                                    ctypes.byref(nnz), ctypes.byref(h), _stream()),
            "spgemm_symbolic")
    return colptr, nnz.value, Plan(h, workspace, A, B, colptr, nnz.value, config, hd)


def spgemm_numeric(plan: Plan, A: CscMatrix, B: CscMatrix, rowidx: Optional[torch.Tensor] = None,
                   values: Optional[torch.Tensor] = None) -> CscMatrix:
    """Rows (ascending) and values of C = A B into new or given buffers."""
    if rowidx is None:
        rowidx = torch.empty(plan.nnz, dtype=torch.int32, device=A.device)
    if values is None:
        values = torch.empty(plan.nnz, dtype=A.dtype, device=A.device)
    N.check(N.lib().spgemm_numeric(plan.handle, ctypes.byref(_csc(A)), ctypes.byref(_csc(B)),
                                   _ptr(plan.colptr), _ptr(rowidx), _ptr(values), _stream()),
            "spgemm_numeric")
    return CscMatrix(A.nrows, B.ncols, plan.colptr, rowidx, values)


def spgemm(A: CscMatrix, B: CscMatrix, config: Optional[Config] = None):
    """C = A B (both phases).  Returns (C, plan)."""
    _, _, plan = spgemm_symbolic(A, B, config)
    C = spgemm_numeric(plan, A, B)
    return C, plan


def single_pass_workspace_size(A: CscMatrix, B: CscMatrix, config: Optional[Config] = None,
                               lib_handle: Optional[Handle] = None) -> int:
    """Workspace bytes of spgemm_single_pass for these patterns (synchronises)."""
    config = replace(config or Config(), dense_cache_bytes=0)
    hd = lib_handle if lib_handle is not None else handle(A.device)
    cA, cB = _csc(A), _csc(B, A.dtype)
    base = workspace_size(A, B, config)
    ws = torch.empty(max(base, 256), dtype=torch.uint8, device=A.device)
    colptr = torch.empty(B.ncols + 1, dtype=torch.int64, device=A.device)
    nbytes = ctypes.c_size_t()
    N.check(N.lib().spgemm_single_pass_size(hd.ptr, ctypes.byref(cA), ctypes.byref(cB),
                                            ctypes.byref(config.native()), _ptr(ws), ws.numel(), _ptr(colptr),
                                            ctypes.byref(nbytes), _stream()), "spgemm_single_pass_size")
    return nbytes.value


def spgemm_single_pass(A: CscMatrix, B: CscMatrix, config: Optional[Config] = None,
                       workspace: Optional[torch.Tensor] = None, lib_handle: Optional[Handle] = None):
    """C = A B without a symbolic phase: every column written to a slot of
    min(Op_j, m) entries, the counts scanned into C's column pointers, then
    the columns copied into C.  Returns (C, plan)."""
    config = config or Config()
    hd = lib_handle if lib_handle is not None else handle(A.device)
    cA, cB = _csc(A), _csc(B, A.dtype)
    if workspace is None:  # a workspace given is checked by the call itself
        need = single_pass_workspace_size(A, B, config, hd)
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=A.device)
    colptr = torch.empty(B.ncols + 1, dtype=torch.int64, device=A.device)
    nnz = ctypes.c_int64()
    h = ctypes.c_void_p()
    N.check(N.lib().spgemm_single_pass(hd.ptr, ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(config.native()),
                                       _ptr(workspace), workspace.numel(), _ptr(colptr), ctypes.byref(nnz),
                                       ctypes.byref(h), _stream()), "spgemm_single_pass")
    plan = Plan(h, workspace, A, B, colptr, nnz.value, config, hd)
    rowidx = torch.empty(nnz.value, dtype=torch.int32, device=A.device)
    values = torch.empty(nnz.value, dtype=A.dtype, device=A.device)
    N.check(N.lib().spgemm_single_pass_copy(plan.handle, _ptr(colptr), _ptr(rowidx), _ptr(values), _stream()),
            "spgemm_single_pass_copy")
    return CscMatrix(A.nrows, B.ncols, colptr, rowidx, values), plan


def _csr(M: CsrMatrix, dtype=None) -> N.SpgCsr:
    dt = dtype if dtype is not None else M.dtype
    for t, want in ((M.rowptr, torch.int64), (M.colidx, torch.int32)):
        if t.dtype != want or not t.is_contiguous() or not t.is_cuda:
            raise TypeError("CSR index arrays must be contiguous CUDA int64 rowptr / int32 colidx")
    return N.SpgCsr(M.nrows, M.ncols, M.nnz, M.rowptr.data_ptr(), _ptr(M.colidx), _ptr(M.values), _DT[dt])


def spgemm_csr(A: CsrMatrix, B: CsrMatrix, config: Optional[Config] = None,
               lib_handle: Optional[Handle] = None):
    """C = A B with A, B and C in CSR (row-wise form).  Returns (C, plan)."""
    config = config or Config()
    hd = lib_handle if lib_handle is not None else handle(A.device)
    cfg = config.native()
    cA, cB = _csr(A), _csr(B, A.dtype)
    nbytes = ctypes.c_size_t()
    N.check(N.lib().spgemm_csr_workspace_size(ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(cfg),
                                              ctypes.byref(nbytes)), "spgemm_csr_workspace_size")
    ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=A.device)
    rowptr = torch.empty(A.nrows + 1, dtype=torch.int64, device=A.device)
    nnz = ctypes.c_int64()
    h = ctypes.c_void_p()
    N.check(N.lib().spgemm_csr_symbolic(hd.ptr, ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(cfg), _ptr(ws),
                                        ws.numel(), _ptr(rowptr), ctypes.byref(nnz), ctypes.byref(h), _stream()),
            "spgemm_csr_symbolic")
    plan = Plan(h, ws, A, B, rowptr, nnz.value, config, hd)
    colidx = torch.empty(nnz.value, dtype=torch.int32, device=A.device)
    values = torch.empty(nnz.value, dtype=A.dtype, device=A.device)
    N.check(N.lib().spgemm_csr_numeric(plan.handle, ctypes.byref(cA), ctypes.byref(cB), _ptr(rowptr),
                                       _ptr(colidx), _ptr(values), _stream()), "spgemm_csr_numeric")
    return CsrMatrix(A.nrows, B.ncols, rowptr, colidx, values), plan


def spgemm_csr_backward(plan: Plan, A: CsrMatrix, B: CsrMatrix, C: CsrMatrix, dC: torch.Tensor):
    """(dA, dB) on the stored entries of CSR A and B for dC on pattern(C)."""
    dA = torch.empty(A.nnz, dtype=A.dtype, device=A.device)
    dB = torch.empty(B.nnz, dtype=A.dtype, device=A.device)
    dC = dC.contiguous()
    N.check(N.lib().spgemm_csr_backward(plan.handle, ctypes.byref(_csr(A)), ctypes.byref(_csr(B)), _ptr(C.rowptr),
                                        _ptr(C.colidx), _ptr(dC), _ptr(dA), _ptr(dB), _stream()),
            "spgemm_csr_backward")
    return dA, dB


def spgemm_backward(plan: Plan, A: CscMatrix, B: CscMatrix, C: CscMatrix, dC: torch.Tensor,
                    need_dA: bool = True, need_dB: bool = True):
    """(dA, dB) on the stored entries of A and B for dC on pattern(C)."""
    dA = torch.empty(A.nnz, dtype=A.dtype, device=A.device) if need_dA else None
    dB = torch.empty(B.nnz, dtype=A.dtype, device=A.device) if need_dB else None
    dC = dC.contiguous()
    N.check(N.lib().spgemm_backward(plan.handle, ctypes.byref(_csc(A)), ctypes.byref(_csc(B)),
                                    _ptr(C.colptr), _ptr(C.rowidx), _ptr(dC), _ptr(dA), _ptr(dB),
                                    _stream()), "spgemm_backward")
    return dA, dB


def csc_transpose(M: CscMatrix, with_perm: bool = True):
    """(M^T as CscMatrix, perm) with T.values = M.values[perm]."""
    cM = _csc(M)
    nbytes = ctypes.c_size_t()
    N.check(N.lib().spg_transpose_workspace_size(ctypes.byref(cM), ctypes.byref(nbytes)),
            "spg_transpose_workspace_size")
    ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=M.device)
    cp = torch.empty(M.nrows + 1, dtype=torch.int64, device=M.device)
    row = torch.empty(M.nnz, dtype=torch.int32, device=M.device)
    vals = torch.empty(M.nnz, dtype=M.dtype, device=M.device) if M.values is not None else None
    perm = torch.empty(M.nnz, dtype=torch.int64, device=M.device) if with_perm else None
    N.check(N.lib().spg_csc_transpose(ctypes.byref(cM), _ptr(cp), _ptr(row), _ptr(vals), _ptr(perm),
                                      _ptr(ws), ws.numel(), _stream()), "spg_csc_transpose")
    return CscMatrix(M.ncols, M.nrows, cp, row, vals), perm


# ------------------------------------------------------------------ batched
class BatchedPlan:
    """Host plan of a batch plus the device workspace and concatenated colptr."""

    def __init__(self, handle, workspace, colptr, nnz, segs, shapes, config, lib_handle=None):
        self._h = handle
        self._lib_handle = lib_handle  # kept alive while the plan is
        self.workspace = workspace
        self.colptr = colptr        # concatenated int64 column pointers
        self.nnz = nnz              # list of nnz(C_i)
        self.segs = segs            # start of product i's column pointers in colptr
        self.shapes = shapes        # (m_i, n_i)
        self.config = config
        self.outputs = None

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def colptr_of(self, i: int) -> torch.Tensor:
        return self.colptr[self.segs[i]:self.segs[i] + self.shapes[i][1] + 1]

    def info(self):
        counts = (ctypes.c_int64 * 64)()
        prod = ctypes.c_int64()
        launches = (ctypes.c_int64 * 3)()
        N.check(N.lib().spg_bplan_info(self.handle, counts, ctypes.byref(prod), launches), "spg_bplan_info")
        return {"bins": list(counts[:14]), "products": prod.value, "launches": list(launches)}

    def check(self) -> None:
        N.check(N.lib().spg_bplan_check(self.handle, _stream()), "spg_bplan_check")

    def destroy(self) -> None:
        if self._h is not None:
            N.lib().spg_bplan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _csc_array(Ms):
    arr = (N.SpgCsc * max(1, len(Ms)))()
    for i, M in enumerate(Ms):
        arr[i] = _csc(M)
    return arr


def spgemm_batched_symbolic(As, Bs, config: Optional[Config] = None) -> BatchedPlan:
    """Column pointers and nnz of every C_i = A_i B_i (synchronises)."""
    if len(As) != len(Bs):
        raise ValueError("A and B lists differ in length")
    config = config or Config()
    cfg = config.native()
    nb = len(As)
    cA, cB = _csc_array(As), _csc_array(Bs)
    nbytes = ctypes.c_size_t()
    N.check(N.lib().spgemm_batched_workspace_size(nb, cA, cB, ctypes.byref(cfg), ctypes.byref(nbytes)),
            "spgemm_batched_workspace_size")
    dev = As[0].device if nb else torch.device("cuda")
    ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    segs, off = [], 0
    for B in Bs:
        segs.append(off)
        off += B.ncols + 1
    colptr = torch.empty(max(off, 1), dtype=torch.int64, device=dev)
    nnz = (ctypes.c_int64 * max(1, nb))()
    h = ctypes.c_void_p()
    hd = handle(dev)
    N.check(N.lib().spgemm_batched_symbolic(hd.ptr, nb, cA, cB, ctypes.byref(cfg), _ptr(ws), ws.numel(),
                                            _ptr(colptr), nnz, ctypes.byref(h), _stream()),
            "spgemm_batched_symbolic")
    shapes = [(A.nrows, B.ncols) for A, B in zip(As, Bs)]
    return BatchedPlan(h, ws, colptr, list(nnz[:nb]), segs, shapes, config, hd)


def spgemm_batched_numeric(plan: BatchedPlan, As, Bs, use_graph: bool = False):
    """All C_i in one persistent launch (optionally a replayed CUDA graph).
    Output buffers are allocated on the first call and reused, so a captured
    graph stays valid across calls."""
    nb = len(As)
    if plan.outputs is None:
        plan.outputs = [(torch.empty(n, dtype=torch.int32, device=A.device),
                         torch.empty(n, dtype=A.dtype, device=A.device)) for n, A in zip(plan.nnz, As)]
    rows = (ctypes.c_void_p * max(1, nb))(*[r.data_ptr() if r.numel() else None for r, _ in plan.outputs])
    vals = (ctypes.c_void_p * max(1, nb))(*[v.data_ptr() if v.numel() else None for _, v in plan.outputs])
    N.check(N.lib().spgemm_batched_numeric(plan.handle, _csc_array(As), _csc_array(Bs), _ptr(plan.colptr), rows,
                                           vals, int(bool(use_graph)), _stream()), "spgemm_batched_numeric")
    return [CscMatrix(A.nrows, B.ncols, plan.colptr_of(i), r, v)
            for i, (A, B, (r, v)) in enumerate(zip(As, Bs, plan.outputs))]


def spgemm_batched(As, Bs, config: Optional[Config] = None, use_graph: bool = False):
    plan = spgemm_batched_symbolic(As, Bs, config)
    return spgemm_batched_numeric(plan, As, Bs, use_graph), plan


def spgemm_batched_backward(plan: BatchedPlan, As, Bs, Cs, dCs, need_dA: bool = True, need_dB: bool = True):
    nb = len(As)
    dA = [torch.empty(A.nnz, dtype=A.dtype, device=A.device) for A in As] if need_dA else None
    dB = [torch.empty(B.nnz, dtype=B.dtype, device=B.device) for B in Bs] if need_dB else None
    rows = (ctypes.c_void_p * max(1, nb))(*[C.rowidx.data_ptr() if C.nnz else None for C in Cs])
    dcs = [d.contiguous() for d in dCs]
    dcp = (ctypes.c_void_p * max(1, nb))(*[d.data_ptr() if d.numel() else None for d in dcs])
    dap = (ctypes.c_void_p * max(1, nb))(*[d.data_ptr() if d.numel() else None for d in dA]) if need_dA else None
    dbp = (ctypes.c_void_p * max(1, nb))(*[d.data_ptr() if d.numel() else None for d in dB]) if need_dB else None
    N.check(N.lib().spgemm_batched_backward(plan.handle, _csc_array(As), _csc_array(Bs), _ptr(plan.colptr), rows,
                                            dcp, dap, dbp, _stream()), "spgemm_batched_backward")
    return dA, dB

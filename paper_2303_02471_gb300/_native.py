"""ctypes view of the C ABI in include/spgemm.h (libspgemm.so, built in-tree).

There is no fallback: if the library is missing or fails to load, every call
raises.  Build it with ``python -m paper_2303_02471_gb300.build`` or
``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspgemm.so")

i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p

SPG_F64, SPG_F32 = 0, 1
SPG_ACC_HASH, SPG_ACC_ESC, SPG_ACC_AUTO = 0, 1, 2
STATUS = {
    0: "SPG_OK", 1: "SPG_ERR_INVALID", 2: "SPG_ERR_WORKSPACE", 3: "SPG_ERR_TABLE_OVERFLOW",
    4: "SPG_ERR_TIMEOUT", 5: "SPG_ERR_CUDA", 6: "SPG_ERR_UNSUPPORTED", 7: "SPG_ERR_INDEX_OVERFLOW",
}
INT64_MAX = (1 << 63) - 1


class SpgCsc(ctypes.Structure):
    _fields_ = [("nrows", i64), ("ncols", i64), ("nnz", i64), ("colptr", vp), ("rowidx", vp),
                ("values", vp), ("dtype", i32)]


class SpgCsr(ctypes.Structure):
    _fields_ = [("nrows", i64), ("ncols", i64), ("nnz", i64), ("rowptr", vp), ("colidx", vp),
                ("values", vp), ("dtype", i32)]


class SpgConfig(ctypes.Structure):
    _fields_ = [("t", i64), ("hash_cta_max", i32), ("cta_threads", i32), ("validate", i32),
                ("table_shrink", i32), ("scratch_cap_bytes", i64), ("dense_cache_bytes", i64),
                ("side_streams", i32), ("test_wait_timeout", i32), ("small_accumulator", i32),
                ("table_slots_pct", i32), ("group_promote", i32)]


class SpgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        super().__init__(f"{where}: {self.name}")


# name -> (restype, argtypes); every symbol include/spgemm.h declares
SIGNATURES = {
    "spg_config_default": (i32, [vp]),
    "spg_status_string": (ctypes.c_char_p, [i32]),
    "spgemm_workspace_size": (i32, [vp, vp, vp, ctypes.POINTER(ctypes.c_size_t)]),
    "spg_create": (i32, [ctypes.POINTER(vp)]),
    "spg_destroy": (i32, [vp]),
    "spgemm_symbolic": (i32, [vp, vp, vp, vp, vp, ctypes.c_size_t, vp, ctypes.POINTER(i64),
                              ctypes.POINTER(vp), vp]),
    "spgemm_numeric": (i32, [vp, vp, vp, vp, vp, vp, vp]),
    "spgemm_single_pass_size": (i32, [vp, vp, vp, vp, vp, ctypes.c_size_t, vp, ctypes.POINTER(ctypes.c_size_t),
                                      vp]),
    "spgemm_single_pass": (i32, [vp, vp, vp, vp, vp, ctypes.c_size_t, vp, ctypes.POINTER(i64),
                                 ctypes.POINTER(vp), vp]),
    "spgemm_single_pass_copy": (i32, [vp, vp, vp, vp, vp]),
    "spgemm_backward": (i32, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "spgemm_csr_workspace_size": (i32, [vp, vp, vp, ctypes.POINTER(ctypes.c_size_t)]),
    "spgemm_csr_symbolic": (i32, [vp, vp, vp, vp, vp, ctypes.c_size_t, vp, ctypes.POINTER(i64),
                                  ctypes.POINTER(vp), vp]),
    "spgemm_csr_numeric": (i32, [vp, vp, vp, vp, vp, vp, vp]),
    "spgemm_csr_backward": (i32, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "spg_plan_check": (i32, [vp, vp]),
    "spg_plan_destroy": (i32, [vp]),
    "spg_plan_info": (i32, [vp, ctypes.POINTER(i32), vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
    "spg_plan_op_counts": (i32, [vp, vp, vp]),
    "spg_plan_bin_stats": (i32, [vp, vp, vp, vp, vp, vp]),
    "spg_plan_launch_count": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
    "spg_plan_bin_streams": (i32, [vp, vp]),
    "spg_plan_set_timing": (i32, [vp, i32]),
    "spg_plan_bin_times": (i32, [vp, vp]),
    "spg_transpose_workspace_size": (i32, [vp, ctypes.POINTER(ctypes.c_size_t)]),
    "spg_csc_transpose": (i32, [vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]),
    "spg_permute_values": (i32, [vp, vp, vp, i64, i32, i32, vp]),
    "spg_csc_transpose_noalloc": (i32, [vp, vp, vp, vp, vp, vp]),
    "spgemm_batched_workspace_size": (i32, [i32, vp, vp, vp, ctypes.POINTER(ctypes.c_size_t)]),
    "spgemm_batched_symbolic": (i32, [vp, i32, vp, vp, vp, vp, ctypes.c_size_t, vp, vp, ctypes.POINTER(vp),
                                      vp]),
    "spgemm_batched_numeric": (i32, [vp, vp, vp, vp, vp, vp, i32, vp]),
    "spgemm_batched_backward": (i32, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "spg_bplan_check": (i32, [vp, vp]),
    "spg_bplan_info": (i32, [vp, vp, ctypes.POINTER(i64), vp]),
    "spg_bplan_destroy": (i32, [vp]),
}

_lib = None


def lib():
    """The loaded library (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is not built; run `python -m paper_2303_02471_gb300.build` "
                "(the CUDA path has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != 0:
        raise SpgError(status, where)

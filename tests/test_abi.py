"""The C ABI without a GPU: the library builds and loads, exports every
function include/spgemm.h declares, and the ctypes layouts match."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spgemm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:spg_status|const char \*)\s*(\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_02471_gb300 import _native, build
    if not os.path.exists(_native.LIB_PATH):
        build.build()
    return _native.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("spg_create", "spg_destroy", "spgemm_symbolic", "spgemm_numeric", "spgemm_backward",
                     "spgemm_batched_symbolic", "spgemm_batched_numeric", "spgemm_batched_backward",
                     "spgemm_workspace_size", "spg_plan_destroy", "spg_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2303_02471_gb300 import _native
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_native.SIGNATURES), set(names) ^ set(_native.SIGNATURES)


def test_struct_layouts():
    from paper_2303_02471_gb300 import _native as N
    assert ctypes.sizeof(N.SpgCsc) == 56 and ctypes.sizeof(N.SpgCsr) == 56
    assert N.SpgCsc.values.offset == 40 and N.SpgCsc.dtype.offset == 48
    assert ctypes.sizeof(N.SpgConfig) == 64
    assert N.SpgConfig.dense_cache_bytes.offset == 32
    assert N.SpgConfig.side_streams.offset == 40 and N.SpgConfig.test_wait_timeout.offset == 44
    assert N.SpgConfig.small_accumulator.offset == 48
    assert N.SpgConfig.table_slots_pct.offset == 52 and N.SpgConfig.group_promote.offset == 56


def test_status_strings_and_defaults(lib):
    from paper_2303_02471_gb300 import _native as N
    for code, name in N.STATUS.items():
        assert lib.spg_status_string(code).decode().startswith(name)
    c = N.SpgConfig()
    assert lib.spg_config_default(ctypes.byref(c)) == 0
    assert c.t == -1 and c.validate == 1 and c.hash_cta_max == 8192
    assert c.side_streams == 1 and c.test_wait_timeout == 0 and c.small_accumulator == N.SPG_ACC_AUTO
    assert c.table_slots_pct == 150 and c.group_promote == 0
    assert lib.spg_config_default(None) == 1


def test_config_range_checks(lib):
    """Out-of-range table sizes and group promotions are rejected before any
    device call (the descriptors are only checked, never read)."""
    from paper_2303_02471_gb300 import _native as N
    M = N.SpgCsc(10, 10, 0, 256, None, None, N.SPG_F64)
    nbytes = ctypes.c_size_t()
    for field, value in (("table_slots_pct", 124), ("table_slots_pct", 401), ("group_promote", -1),
                         ("group_promote", 3)):
        c = N.SpgConfig()
        assert lib.spg_config_default(ctypes.byref(c)) == 0
        setattr(c, field, value)
        assert lib.spgemm_workspace_size(ctypes.byref(M), ctypes.byref(M), ctypes.byref(c),
                                         ctypes.byref(nbytes)) == 1, (field, value)
    c = N.SpgConfig()
    lib.spg_config_default(ctypes.byref(c))
    c.table_slots_pct, c.group_promote = 400, 2
    # valid: passes the checks (and fails only for want of a GPU on a CPU machine)
    assert lib.spgemm_workspace_size(ctypes.byref(M), ctypes.byref(M), ctypes.byref(c), ctypes.byref(nbytes)) != 1


def test_host_only_calls(lib):
    from paper_2303_02471_gb300 import _native as N
    M = N.SpgCsc(10, 7, 30, None, None, None, 0)
    nbytes = ctypes.c_size_t()
    assert lib.spg_transpose_workspace_size(ctypes.byref(M), ctypes.byref(nbytes)) == 0
    assert nbytes.value >= 30 * 8
    bad = N.SpgCsc(-1, 7, 30, None, None, None, 0)
    assert lib.spg_transpose_workspace_size(ctypes.byref(bad), ctypes.byref(nbytes)) == 1
    assert lib.spg_plan_destroy(None) == 0
    assert lib.spg_destroy(None) == 0
    assert lib.spg_create(None) == 1
    assert lib.spg_bplan_destroy(None) == 0
    assert lib.spg_plan_check(None, None) == 1
    assert lib.spg_permute_values(None, None, None, 0, 0, 0, None) == 0
    assert lib.spg_permute_values(None, None, None, 5, 0, 0, None) == 1


def _batch_bytes(lib, shapes, cache):
    # shapes only: the pointers are never dereferenced on the host
    from paper_2303_02471_gb300 import _native as N
    As = (N.SpgCsc * len(shapes))()
    Bs = (N.SpgCsc * len(shapes))()
    for i, (m, k, n) in enumerate(shapes):
        As[i] = N.SpgCsc(m, k, 4 * k, 16, 16, 16, 0)
        Bs[i] = N.SpgCsc(k, n, 4 * n, 16, 16, 16, 0)
    c = N.SpgConfig()
    lib.spg_config_default(ctypes.byref(c))
    if cache is not None:
        c.dense_cache_bytes = cache
    nbytes = ctypes.c_size_t()
    assert lib.spgemm_batched_workspace_size(len(shapes), As, Bs, ctypes.byref(c), ctypes.byref(nbytes)) == 0
    return nbytes.value


def test_batched_workspace_holds_the_kept_dense_flags(lib):
    """Kept flags of per-warp dense columns: every column's flags (n_i words
    of ceil(m_i / 32)) up to dense_cache_bytes, and none when a product has
    more than 32768 rows (its dense columns run one per CTA)."""
    small = [(1000, 300, 500), (32768, 200, 90)]
    words = 500 * 32 + 90 * 1024
    base = _batch_bytes(lib, small, 0)
    full = _batch_bytes(lib, small, None)
    # the cache and the column offsets, each padded to 256 bytes
    assert words * 4 <= full - base <= words * 4 + (590 + 1) * 8 + 512
    capped = _batch_bytes(lib, small, 4096)
    assert 4096 <= capped - base <= 4096 + (590 + 1) * 8 + 512
    tall = small + [(32769, 10, 10)]
    assert _batch_bytes(lib, tall, None) == _batch_bytes(lib, tall, 0)

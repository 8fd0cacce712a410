"""CPU checks of the C ABI: the library builds, loads, exports every function
include/psort.h declares, and rejects bad arguments before touching a GPU."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_05245_gb300 import _lib, build
    build.build()
    return _lib.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "psort.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|void)\s+(ps_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_function(lib):
    names = header_functions()
    assert "ps_sort" in names and "ps_sort_pairs" in names
    for n in names:
        assert hasattr(lib, n), "libpsort.so does not export %s" % n
    from paper_2305_05245_gb300 import _lib
    assert sorted(_lib.EXPORTS) == sorted(n for n in names if n in _lib.EXPORTS)


def test_status_strings(lib):
    assert lib.ps_status_string(0) == b"ok"
    for s in range(-7, 0):
        assert lib.ps_status_string(s) and lib.ps_status_string(s) != b"unknown status"
    assert lib.ps_status_string(-99) == b"unknown status"


def test_argument_errors_without_gpu(lib):
    from paper_2305_05245_gb300 import _lib
    p = _lib.PsParams()
    # negative size, bad dtype, bad mode, params out of range
    assert lib.ps_sort(None, -1, 0, 0, None) == -1
    assert lib.ps_sort(None, 10, 9, 0, None) == -2
    assert lib.ps_sort(None, 10, 0, 7, None) == -2
    p.n_blocks = 5000
    assert lib.ps_sort_ex(None, 10, 0, 1, ctypes.byref(p), None, None) == -1
    p.n_blocks, p.n_parts = 4, (1 << 20) + 1
    assert lib.ps_sort_ex(None, 10, 0, 1, ctypes.byref(p), None, None) == -1
    p.n_parts = 4
    # launch shapes: unknown values are invalid, unoffered combinations unsupported
    for it, th in [(8, 256), (24, 0), (0, 64), (32, 1024), (-16, 256)]:
        p.items_per_thread, p.block_threads = it, th
        assert lib.ps_sort_ex(None, 10, 0, 1, ctypes.byref(p), None, None) == -1, (it, th)
    for it, th in [(32, 512), (32, 0), (0, 128)]:
        p.items_per_thread, p.block_threads = it, th
        assert lib.ps_sort_pairs(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 10, 0,
                                 ctypes.byref(p), None, None) == -2, (it, th)
    p.items_per_thread, p.block_threads = 0, 0
    p.merge_variant = 3
    assert lib.ps_sort_ex(None, 10, 0, 1, ctypes.byref(p), None, None) == -1
    p.merge_variant = -1
    assert lib.ps_sort_ex(None, 10, 0, 1, ctypes.byref(p), None, None) == -1
    # null keys with n >= 2, misaligned keys
    assert lib.ps_sort(None, 10, 0, 0, None) == -1
    assert lib.ps_sort(ctypes.c_void_p(0x1002), 10, 1, 0, None) == -1
    assert lib.ps_sort_pairs(ctypes.c_void_p(0x1000), None, 10, 0, None, None, None) == -1
    # records sorted by an embedded key: size, record size, key offset, mode, alignment
    assert lib.ps_sort_struct(None, -1, 16, 0, 1, None, None) == -1
    assert lib.ps_sort_struct(None, 1 << 32, 16, 0, 1, None, None) == -1
    assert lib.ps_sort_struct(None, 10, 12, 0, 1, None, None) == -1
    assert lib.ps_sort_struct(None, 10, 0, 0, 1, None, None) == -1
    assert lib.ps_sort_struct(None, 10, _lib.PS_STRUCT_MAX_BYTES + 8, 0, 1, None, None) == -1
    assert lib.ps_sort_struct(None, 10, 16, 4, 1, None, None) == -1
    assert lib.ps_sort_struct(None, 10, 16, 16, 1, None, None) == -1
    assert lib.ps_sort_struct(None, 10, 16, 8, 5, None, None) == -2
    assert lib.ps_sort_struct(None, 10, 16, 8, 1, None, None) == -1
    assert lib.ps_sort_struct(ctypes.c_void_p(0x1004), 10, 16, 8, 1, None, None) == -1
    assert lib.ps_sort_struct(None, 1, 96, 0, 0, None, None) == 0
    # n = 0 and n = 1 are no-ops
    assert lib.ps_sort(None, 0, 0, 0, None) == 0
    assert lib.ps_sort(None, 1, 3, 1, None) == 0
    assert lib.ps_sort_host(None, 1, 0, 0, None, None) == 0
    assert lib.ps_sort_host(None, 5, 0, 0, None, None) == -1


def test_autotune_table_without_gpu(lib):
    """ps_autotune's argument checks and the tuned table's get/set (no GPU)."""
    from paper_2305_05245_gb300 import _lib
    p = _lib.PsParams()
    assert lib.ps_autotune(-1, 1, 1 << 14, 1 << 16, 0, None) == -2
    assert lib.ps_autotune(0, 9, 1 << 14, 1 << 16, 0, None) == -2
    assert lib.ps_autotune(0, 1, 1, 1 << 16, 0, None) == -1
    assert lib.ps_autotune(0, 1, 1 << 16, 1 << 14, 0, None) == -1
    assert lib.ps_autotune(0, 1, 1 << 14, 1 << 16, 2, None) == -1
    assert lib.ps_autotune_get(0, 0, 40, ctypes.byref(p)) == -7
    assert lib.ps_autotune_get(9, 0, 40, ctypes.byref(p)) == -2
    p.n_blocks, p.n_parts = 5000, 4
    assert lib.ps_autotune_set(0, 0, 40, ctypes.byref(p)) == -1
    p.n_blocks, p.n_parts = 48, 96
    assert lib.ps_autotune_set(2, 0, 40, ctypes.byref(p)) == 0   # float32 shares the 32-bit entry
    q = _lib.PsParams()
    assert lib.ps_autotune_get(4, 0, 40, ctypes.byref(q)) == 0 and (q.n_blocks, q.n_parts) == (48, 96)
    assert lib.ps_autotune_get(1, 0, 40, ctypes.byref(q)) == -7  # 64-bit keys: separate entry
    assert lib.ps_autotune_get(0, 1, 40, ctypes.byref(q)) == -7  # batched table: separate
    r = _lib.PsParams()
    assert lib.ps_resolve_params(1 << 40, 0, None, ctypes.byref(r)) == 0
    assert (r.n_blocks, r.n_parts) == (48, 96)
    r2 = _lib.PsParams()
    r2.n_blocks = 64
    assert lib.ps_resolve_params(1 << 40, 0, ctypes.byref(r2), ctypes.byref(r)) == 0
    assert r.n_blocks == 64  # explicit fields win
    # an entry carries a launch shape too; it applies when n_blocks and the
    # shape are automatic, and unoffered or invalid shapes are refused
    p.items_per_thread, p.block_threads = 16, 512
    assert lib.ps_autotune_set(0, 0, 40, ctypes.byref(p)) == 0
    assert lib.ps_autotune_get(0, 0, 40, ctypes.byref(q)) == 0
    assert (q.n_blocks, q.n_parts, q.items_per_thread, q.block_threads) == (48, 96, 16, 512)
    assert lib.ps_resolve_params(1 << 40, 0, None, ctypes.byref(r)) == 0
    assert (r.items_per_thread, r.block_threads) == (16, 512)
    assert lib.ps_resolve_params(1 << 40, 0, ctypes.byref(r2), ctypes.byref(r)) == 0
    assert (r.items_per_thread, r.block_threads) == (0, 0)  # explicit n_B: automatic shape
    p.items_per_thread, p.block_threads = 24, 512
    assert lib.ps_autotune_set(0, 0, 40, ctypes.byref(p)) == -1
    assert lib.ps_autotune_set(0, 0, 40, None) == 0
    assert lib.ps_autotune_get(0, 0, 40, ctypes.byref(q)) == -7


def test_injected_allocation_failure_without_gpu(lib):
    """An allocation failure (injected on the host) surfaces as
    PS_ERR_NO_MEMORY from every entry point that allocates, before any device
    work; the injection wears off after the given count."""
    from paper_2305_05245_gb300 import _lib
    fake = ctypes.c_void_p(0x10000)  # never touched: the sort stops at its first allocation
    assert lib.ps_debug_fail_alloc(-1) == -1
    assert lib.ps_debug_fail_alloc(3) == 0
    try:
        assert lib.ps_sort(fake, 1 << 20, 1, 1, None) == -3
        assert lib.ps_sort_pairs(fake, fake, 1 << 20, 1, None, None, None) == -3
        rec = ctypes.c_void_p(0x20000)
        assert lib.ps_sort_struct(rec, 1000, 16, 0, 1, None, None) == -3
    finally:
        assert lib.ps_debug_fail_alloc(0) == 0


def test_default_parameter_table_without_gpu(lib):
    """Automatic parameters: the measured table for 2^14..2^31 keys (one block
    and one partition up to 2^19), the size heuristic beyond; explicit fields
    are kept; the allocation-free path is independent of the table."""
    import paper_2305_05245_gb300 as ps
    for b in range(14, 20):
        assert ps.resolve_params(1 << b, 1) == (1, 1)
        assert ps.resolve_params(1 << b, 0) == (1, 1)
    assert ps.resolve_params(1 << 30, 1) == (64, 128)
    assert ps.resolve_params(1 << 30, 3) == (64, 128)   # float64 shares the 64-bit table
    assert ps.resolve_params(1 << 26, 2) == ps.resolve_params(1 << 26, 0)
    nb, np_ = ps.resolve_params(1 << 36, 1)             # beyond the table: the heuristic
    assert nb == 1024 and np_ == 256
    assert ps.resolve_params(1 << 30, 1, n_blocks=7) == (7, 7)
    assert ps.resolve_params(1 << 30, 1, n_parts=5)[1] == 5
    nb, np_ = ps.resolve_params(1 << 30, -1)            # records: heuristic
    assert 1 <= nb <= 4096 and 1 <= np_ <= 256


def test_resolve_and_workspace(lib):
    import paper_2305_05245_gb300 as ps
    nb, np_ = ps.resolve_params(1 << 26, 0)
    assert 1 <= nb <= 4096 and 1 <= np_ <= (1 << 20)
    assert ps.resolve_params(1 << 20, 0, 64, 64) == (64, 64)
    w32 = ps.workspace_bytes(1 << 20, 0, 64, 64)
    w64 = ps.workspace_bytes(1 << 20, 1, 64, 64)
    assert w32 >= 4 << 20 and w64 >= 8 << 20 and w64 > w32
    assert ps.workspace_bytes(1, 0) == 0

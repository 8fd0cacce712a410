"""ps_sort_noalloc, the entry point for callers that may not allocate device
memory (for example code that runs while someone else captures a CUDA graph,
real-time loops that forbid allocator calls, or hosts whose device memory
pools belong to another runtime).  It must give exactly the sorted result --
the oracle's plain definition, and the ordinary entry point's output -- call
after call, although every call reuses the same static scratch array.  This
file is collected last on purpose."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import synth

CODES = {"int32": 0, "int64": 1, "float32": 2, "float64": 3, "uint32": 4, "uint64": 5}


def _lib():
    from paper_2305_05245_gb300 import _lib, build
    build.build()
    return _lib.load(), _lib


def test_rejects_sizes_beyond_the_static_scratch():
    lib, L = _lib()
    # rejected before any device work is queued, so no GPU is needed here
    assert lib.ps_sort_noalloc(ctypes.c_void_p(0x1000), L.PS_NOALLOC_MAX_KEYS + 1, 1, 1, None) == -1
    assert lib.ps_sort_noalloc(None, 0, 0, 0, None) == 0
    assert lib.ps_sort_noalloc(None, 1, 0, 0, None) == 0
    assert lib.ps_sort_noalloc(ctypes.c_void_p(0x1000), 10, 9, 0, None) == -2


def test_largest_shape_fits_the_static_scratch():
    """At PS_NOALLOC_MAX_KEYS keys the size heuristic chooses 4 blocks and 4
    partitions; that sort's workspace must fit the static array for 4- and
    8-byte keys alike."""
    lib, L = _lib()
    p = L.PsParams(4, 4, 0, 0)
    for code in (CODES["int32"], CODES["int64"]):
        need = ctypes.c_size_t(0)
        assert lib.ps_workspace_bytes(L.PS_NOALLOC_MAX_KEYS, code, ctypes.byref(p), ctypes.byref(need)) == 0
        assert need.value <= L.PS_NOALLOC_SCRATCH_BYTES, (code, need.value)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,n,mode", [("int32", 1_000_003 // 3, 1), ("float64", 1 << 20, 0),
                                          ("int64", 1 << 20, 1), ("uint32", 4097, 0)])
def test_noalloc_matches_oracle_and_ps_sort_twice(ora, dtype, n, mode):
    import torch
    lib, L = _lib()
    code = CODES[dtype]
    stream = torch.cuda.current_stream().cuda_stream or None
    for call in range(2):  # two calls in a row share (and overwrite) the scratch array
        keys = synth.keys(n, dtype, "few_unique" if call else "uniform",
                          seed=synth.seed_for("noalloc", dtype, call))
        raw = keys.view(np.int32 if keys.itemsize == 4 else np.int64)
        a = torch.from_numpy(raw.copy()).cuda()
        b = torch.from_numpy(raw.copy()).cuda()
        rc = lib.ps_sort_noalloc(ctypes.c_void_p(a.data_ptr()), n, code, mode, stream)
        assert rc == 0, "ps_sort_noalloc returned %d" % rc
        rc = lib.ps_sort_ex(ctypes.c_void_p(b.data_ptr()), n, code, mode, None, None, stream)
        assert rc == 0
        torch.cuda.synchronize()
        got = a.cpu().numpy().view(keys.dtype)
        want = ora.reference_sort(keys)
        assert got.tobytes() == want.tobytes(), "call %d: ps_sort_noalloc differs from the oracle" % call
        assert torch.equal(a, b), "call %d: ps_sort_noalloc differs from ps_sort_ex" % call


@pytest.mark.gpu
def test_noalloc_sorts_while_allocation_fails(ora):
    """With every library allocation failing (host-side injection), the
    allocating entry point reports PS_ERR_NO_MEMORY while ps_sort_noalloc
    still sorts exactly: it never asks for memory."""
    import torch
    lib, L = _lib()
    n = 300_001
    keys = synth.keys(n, "int64", "uniform", seed=synth.seed_for("noalloc", "inject"))
    a = torch.from_numpy(keys.copy()).cuda()
    b = torch.from_numpy(keys.copy()).cuda()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream or None
    assert lib.ps_debug_fail_alloc(1000) == 0
    try:
        assert lib.ps_sort_noalloc(ctypes.c_void_p(a.data_ptr()), n, CODES["int64"], 1, stream) == 0
        # the injection is armed: the ordinary path fails before queueing anything
        assert lib.ps_sort_ex(ctypes.c_void_p(b.data_ptr()), n, CODES["int64"], 1, None, None, stream) == -3
    finally:
        assert lib.ps_debug_fail_alloc(0) == 0
    torch.cuda.synchronize()
    assert a.cpu().numpy().tobytes() == ora.reference_sort(keys).tobytes()
    assert torch.equal(b.cpu(), torch.from_numpy(keys)), "a failed sort must leave its keys untouched"

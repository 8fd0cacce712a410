"""ps_sort_noalloc, the entry point for callers that may not allocate device
memory (for example code that runs while someone else captures a CUDA graph,
or hosts whose device memory pools belong to another runtime).  It must give
exactly the result of the ordinary entry point, call after call, although
every call reuses the same static scratch array.  This file is collected last
on purpose."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import synth


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


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,n,mode", [("int32", 1_000_003 // 3, 1), ("float64", 1 << 20, 0),
                                          ("int64", 1 << 20, 1), ("uint32", 4097, 0)])
def test_noalloc_matches_ps_sort_twice(dtype, n, mode):
    import torch
    lib, L = _lib()
    code = {"int32": 0, "int64": 1, "float32": 2, "float64": 3, "uint32": 4, "uint64": 5}[dtype]
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
        assert torch.equal(a, b), "call %d: ps_sort_noalloc differs from ps_sort_ex" % call

"""ps_sort_host: keys in host memory, pageable (copied in and out) or pinned
and mapped (read by the first pass and written by the last pass directly),
against the oracle's plain definition of the result."""
from __future__ import annotations

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_05245_gb300 as ps
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ps


CASES = [
    # (n, dtype, dist, n_B, n_P): 0 = automatic
    (5_000, "int32", "uniform", 1, 1),          # one tile: the tile sort writes the result
    (5_000, "float64", "gaussian", 0, 0),
    (100_003, "int64", "few_unique", 4, 4),
    (300_007, "float32", "uniform", 1, 1),      # one block, in-block passes only
    (1_000_003, "uint64", "uniform", 0, 0),
    (3_000_017, "int32", "reverse", 2, 8),
    (2_000_000, "float64", "uniform", 0, 0),
    # 2^24 keys and more in pinned memory take the pipelined path: blocks copied
    # in groups while earlier groups are block-sorted, then steps 2 to 4
    ((1 << 24) + 12_345, "int64", "uniform", 0, 0),
    (20_000_003, "float32", "gaussian", 48, 96),
    ((1 << 24) + 1, "int32", "few_unique", 7, 3),
]


@pytest.mark.parametrize("mode", ["regular", "exact"])
@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("n,dtype,dist,n_B,n_P", CASES)
def test_sort_host(ps, ora, n, dtype, dist, n_B, n_P, pinned, mode):
    import torch
    if dist == "gaussian" and not dtype.startswith("float"):
        pytest.skip("gaussian keys are floating point")
    if n >= (1 << 24) and not pinned:
        pytest.skip("large cases are for the pinned (pipelined) path")
    keys = synth.keys(n, dtype, dist, seed=synth.seed_for("host", n, dtype, dist))
    want = ora.reference_sort(keys)
    if pinned:
        t = torch.from_numpy(keys.view({4: np.int32, 8: np.int64}[keys.itemsize]).copy()).pin_memory()
        if dtype.startswith("uint"):
            import ctypes
            from paper_2305_05245_gb300 import _lib
            lib = _lib.load()
            rc = lib.ps_sort_host(t.data_ptr(), n, {"uint32": 4, "uint64": 5}[dtype], ps._mode(mode),
                                  ctypes.byref(ps._params(n_B, n_P)), None)
            _lib.check(lib, "ps_sort_host", rc)
        else:
            ps.sort_host(t.view(getattr(torch, dtype)), mode, n_B, n_P)
        got = t.numpy().view(keys.dtype)
    else:
        got = keys.copy()
        ps.sort_host(got, mode, n_B, n_P)
    assert got.tobytes() == want.tobytes()


def test_sort_host_oracle_steps(ps, ora):
    """A pinned, mapped input through the full step-by-step oracle."""
    import torch
    n, nb, np_ = 700_001, 16, 16
    keys = synth.keys(n, "int64", "three_valued", seed=synth.seed_for("host-oracle"))
    t = torch.from_numpy(keys.copy()).pin_memory()
    ps.sort_host(t, "exact", nb, np_)
    ref = ora.sort(keys, 1, nb, np_)
    assert t.numpy().tobytes() == ref.out.tobytes()


def test_sort_host_misaligned(ps):
    buf = np.zeros(101, dtype=np.int64)
    view = buf.view(np.uint8)[4:4 + 8 * 100]
    import ctypes
    from paper_2305_05245_gb300 import _lib
    lib = _lib.load()
    assert lib.ps_sort_host(ctypes.c_void_p(view.ctypes.data), 100, 1, 1, None, None) == -1

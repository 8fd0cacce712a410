"""GPU parity of every launch shape (ps_params items_per_thread x
block_threads): the tile sort and the chunk merges compiled for each shape
must give the oracle's output and intermediates element by element.  Sizes
span several tiles of the shape, one in-block merge pass, the final merge and
a ragged tail; both pivot modes; 32- and 64-bit keys, float keys included."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from test_gpu_parity import MODES, assert_parity  # noqa: F401  (shared oracle comparison)

pytestmark = pytest.mark.gpu

SHAPES = [(16, 128), (16, 256), (16, 512), (32, 128), (32, 256), (32, 512)]


@pytest.fixture(scope="module")
def ps():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_05245_gb300 as ps
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ps


def _run(ps, keys, mode, n_B, n_P, items, threads):
    import torch
    x = torch.from_numpy(keys.view(np.int32 if keys.itemsize == 4 else np.int64).copy()).cuda()
    x = x.view({np.dtype(np.int32): torch.int32, np.dtype(np.int64): torch.int64,
                np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64}[keys.dtype])
    tr = ps.sort(x, mode, n_blocks=n_B, n_parts=n_P, trace=True, items_per_thread=items, block_threads=threads)
    torch.cuda.synchronize()
    out = x.cpu().numpy().view(keys.dtype)
    t = {"pivots": tr.pivots.cpu().numpy().view(keys.dtype)[: max(n_P - 1, 0)],
         "pivot_payload": None, "c": tr.c.cpu().numpy()[: max(n_P - 1, 0)],
         "splits": tr.splits.cpu().numpy(), "offsets": tr.offsets.cpu().numpy()}
    return out, t


@pytest.mark.parametrize("mode", ["regular", "exact"])
@pytest.mark.parametrize("dtype,dist", [("int64", "uniform"), ("int32", "few_unique"),
                                        ("float64", "gaussian"), ("float32", "uniform")])
@pytest.mark.parametrize("items,threads", SHAPES)
def test_shape_parity(ps, ora, items, threads, dtype, dist, mode):
    tile = items * threads
    n = 9 * tile + 1234            # blocks of about 3 tiles: one in-block pass
    keys = synth.keys(n, dtype, dist, seed=synth.seed_for("launch-shape", items, threads, dtype, dist))
    out, t = _run(ps, keys, mode, 3, 5, items, threads)
    assert_parity(ora, keys, mode, 3, 5, out, None, t)


@pytest.mark.parametrize("items,threads", [(16, 128), (32, 512)])
def test_shape_wide_final_merge(ps, ora, items, threads):
    """64 blocks of one tile and a ragged last one: fan-in 64 in step 4."""
    n = 64 * items * threads - 777
    keys = synth.keys(n, "int64", "uniform", seed=synth.seed_for("launch-shape-wide", items, threads))
    for mode in ("regular", "exact"):
        out, t = _run(ps, keys, mode, 64, 16, items, threads)
        assert_parity(ora, keys, mode, 64, 16, out, None, t)


def test_shape_records_only_automatic(ps):
    """Records offer only their automatic shape."""
    import torch
    from paper_2305_05245_gb300 import PsortError
    k = torch.zeros(1000, dtype=torch.int64, device="cuda")
    p = torch.zeros(1000, dtype=torch.int32, device="cuda")
    import ctypes
    from paper_2305_05245_gb300 import _lib
    lib = _lib.load()
    prm = ps._params(0, 0, "tree", 32, 512)
    assert lib.ps_sort_pairs(k.data_ptr(), p.data_ptr(), 1000, 1, ctypes.byref(prm), None, None) == -2
    prm = ps._params(0, 0, "tree", 16, 256)
    assert lib.ps_sort_pairs(k.data_ptr(), p.data_ptr(), 1000, 1, ctypes.byref(prm), None, None) == 0
    torch.cuda.synchronize()
    with pytest.raises(PsortError):
        ps.sort(torch.zeros(10, dtype=torch.int32, device="cuda"), "exact", items_per_thread=24)

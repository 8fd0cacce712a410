"""Step 4's three chunk-merge variants (pairwise merge levels, copy and sort,
selection tree; Sec. 2.2 and Sec. 4's comparison of multiway merging) give
the oracle's output and intermediates on the same inputs."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from test_gpu_parity import MODES, assert_parity

pytestmark = pytest.mark.gpu

SHAPES = [
    # (n, dtype, dist, n_B, n_P)
    (2, "int32", "uniform", 2, 1), (1000, "int32", "few_unique", 3, 7),
    (50_001, "float32", "few_unique", 13, 7), (100_003, "uint64", "three_valued", 16, 16),
    (300_007, "float64", "gaussian", 64, 64), (1_000_003, "int64", "uniform", 100, 3),
    (77, "int32", "uniform", 100, 9), (12_345, "float64", "few_unique", 4096, 2),
    (2_000_003, "int32", "uniform", 256, 200), (3_000_000, "int64", "almost_sorted", 48, 48),
]


@pytest.fixture(scope="module")
def ps():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_05245_gb300 as ps
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ps


def _run(ps, keys, mode, n_B, n_P, variant):
    import torch
    x = torch.from_numpy(keys.view({4: np.int32, 8: np.int64}[keys.itemsize]).copy()).cuda()
    if keys.dtype in (np.float32, np.float64):
        x = x.view(torch.float32 if keys.dtype == np.float32 else torch.float64)
    if keys.dtype in (np.uint32, np.uint64):
        import ctypes
        from paper_2305_05245_gb300 import _lib
        lib = _lib.load()
        code = 4 if keys.dtype == np.uint32 else 5
        tr, ct = ps._make_trace(x.numel(), code, n_B, n_P, x.dtype, x.device, False)
        rc = lib.ps_sort_ex(x.data_ptr(), x.numel(), code, ps._mode(mode),
                            ctypes.byref(ps._params(n_B, n_P, variant)), ctypes.byref(ct), ps._stream_handle(None))
        _lib.check(lib, "ps_sort_ex", rc)
    else:
        tr = ps.sort(x, mode, n_blocks=n_B, n_parts=n_P, trace=True, merge_variant=variant)
    torch.cuda.synchronize()
    out = x.cpu().numpy().view(keys.dtype)
    t = {"pivots": tr.pivots.cpu().numpy().view(keys.dtype)[: max(n_P - 1, 0)],
         "c": tr.c.cpu().numpy()[: max(n_P - 1, 0)], "splits": tr.splits.cpu().numpy(),
         "offsets": tr.offsets.cpu().numpy()}
    return out, t


@pytest.mark.parametrize("variant", ["sort", "select"])
@pytest.mark.parametrize("mode", ["regular", "exact"])
@pytest.mark.parametrize("n,dtype,dist,n_B,n_P", SHAPES)
def test_variant_parity(ps, ora, n, dtype, dist, n_B, n_P, mode, variant):
    keys = synth.keys(n, dtype, dist, seed=synth.seed_for("variant", n, dtype, dist))
    out, t = _run(ps, keys, mode, n_B, n_P, variant)
    assert_parity(ora, keys, mode, n_B, n_P, out, None, t)


@pytest.mark.parametrize("variant", ["tree", "sort", "select"])
def test_variant_records(ps, ora, variant):
    """Records (uint64 key, uint32 payload) under each variant."""
    import torch
    n, n_B, n_P = 200_003, 24, 24
    k, p = synth.records(n, seed=synth.seed_for("variant-rec"), dist="few_unique")
    x = torch.from_numpy(k.view(np.int64).copy()).cuda()
    y = torch.from_numpy(p.view(np.int32).copy()).cuda()
    ps.sort_pairs(x, y, "exact", n_blocks=n_B, n_parts=n_P, merge_variant=variant)
    torch.cuda.synchronize()
    ref = ora.sort(k, MODES["exact"], n_B, n_P, payload=p)
    assert np.array_equal(x.cpu().numpy().view(np.uint64), ref.out)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), ref.out_payload)


def test_variant_default_size(ps):
    """2^26 int64 with automatic parameters: the three variants agree."""
    import torch
    base = synth.keys_torch(1 << 26, "int64", "uniform", seed=synth.seed_for("variant-2p26"))
    outs = []
    for v in ("tree", "sort", "select"):
        x = base.clone()
        ps.sort(x, "exact", merge_variant=v)
        outs.append(x)
    torch.cuda.synchronize()
    assert bool((outs[0][1:] >= outs[0][:-1]).all())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])

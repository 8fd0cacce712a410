"""ps_sort_batch: every segment of a batch must come out exactly as the
method sorts it alone (the unique sorted permutation), whatever the mix of
segment lengths -- empty, one key, one tile, several tiles, several blocks."""
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
    assert torch.cuda.is_available()
    return ps


def make_batch(n_segs, max_log, dtype, dist, seed, special=()):
    z = synth.splitmix64(seed, n_segs)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    lens = np.floor(2.0 ** (u * max_log)).astype(np.int64) - 1
    lens[: len(special)] = special
    offs = np.zeros(n_segs + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    keys = synth.keys(int(offs[-1]), dtype, dist, seed=seed + 1)
    return keys, offs


def reference(ora, keys, offs):
    """Each segment sorted alone (plain definition: stable argsort on the order
    key within each segment)."""
    seg = np.repeat(np.arange(len(offs) - 1), np.diff(offs))
    idx = np.lexsort((ora.order_key(keys), seg))
    return keys[idx]


def to_dev(a):
    import torch
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32).copy()).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64).copy()).cuda()
    return torch.from_numpy(a.copy()).cuda()


SPECIAL = [0, 1, 2, 1023, 1024, 1025, 8191, 8192, 8193, 16385, 70_000, 300_001, 1 << 20]


@pytest.mark.parametrize("dtype,dist", [("int32", "uniform"), ("int64", "few_unique"),
                                        ("float32", "gaussian"), ("float64", "uniform"),
                                        ("uint32", "three_valued"), ("int64", "sorted")])
@pytest.mark.parametrize("mode", ["regular", "exact"])
def test_batch_matches_reference(ps, ora, dtype, dist, mode):
    import torch
    keys, offs = make_batch(600, 17, dtype, dist, seed=synth.seed_for("batch", dtype, dist) % 100000,
                            special=SPECIAL)
    x = to_dev(keys)
    if dtype == "uint32":
        from paper_2305_05245_gb300 import _lib
        import ctypes
        o = torch.from_numpy(offs).cuda()
        rc = _lib.load().ps_sort_batch(ctypes.c_void_p(o.data_ptr()), len(offs) - 1,
                                       ctypes.c_void_p(x.data_ptr()), 4, 1 if mode == "exact" else 0, None)
        assert rc == 0
    else:
        ps.sort_batch(x, torch.from_numpy(offs).cuda(), mode)
    torch.cuda.synchronize()
    got = x.cpu().numpy().view(keys.dtype)
    want = reference(ora, keys, offs)
    assert got.tobytes() == want.tobytes()


def test_batch_equals_per_segment_sort(ps):
    import torch
    keys, offs = make_batch(60, 19, "int64", "uniform", seed=7, special=[8193, 1 << 18, 3])
    x = to_dev(keys)
    ps.sort_batch(x, torch.from_numpy(offs).cuda(), "exact")
    y = to_dev(keys)
    for i in range(len(offs) - 1):
        seg = y[offs[i]:offs[i + 1]]
        if seg.numel() > 1:
            ps.sort(seg, "exact")
    torch.cuda.synchronize()
    assert torch.equal(x, y)


@pytest.mark.parametrize("dtype", ["int32", "float64"])
def test_batch_many_tiny_segments(ps, ora, dtype):
    """100,000 segments of 2..64 keys (the small-segment bin: a warp per
    segment in the persistent front kernel, many work items per CTA) plus a
    few at the bin edges."""
    import torch
    z = synth.splitmix64(synth.seed_for("tiny", dtype), 100_000)
    lens = (2 + (z % np.uint64(63))).astype(np.int64)
    lens[:4] = [1024, 1025, 1, 0]
    offs = np.zeros(len(lens) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    keys = synth.keys(int(offs[-1]), dtype, "few_unique", seed=synth.seed_for("tiny-keys", dtype))
    x = to_dev(keys)
    ps.sort_batch(x, torch.from_numpy(offs).cuda(), "exact")
    torch.cuda.synchronize()
    assert x.cpu().numpy().tobytes() == reference(ora, keys, offs).tobytes()


@pytest.mark.parametrize("dtype,lens", [
    ("int64", [1024] * 700 + [2, 3, 31, 32, 33, 1000]),          # warp items only
    ("uint32", [8192, 1025, 4097, 2048, 7777] * 200),            # tile items only
    ("float32", [2, 8192, 1024, 1025, 5000, 17] * 150),          # both, interleaved
    ("uint64", [1, 0, 1024, 0, 8192, 1] * 100),                  # empty and one-key segments between
])
def test_batch_front_kernel(ps, ora, dtype, lens):
    """The persistent front kernel (every segment of at most one tile): one
    launch per batch, whatever the mix of warp and tile items, and every
    segment equal to the oracle's plain sorted result."""
    import ctypes
    import torch
    from paper_2305_05245_gb300 import _lib
    lens = np.array(lens, dtype=np.int64)
    offs = np.zeros(len(lens) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    dist = "gaussian" if dtype.startswith("float") else "few_unique"
    keys = synth.keys(int(offs[-1]), dtype, dist, seed=synth.seed_for("front", dtype))
    x = to_dev(keys)
    o = torch.from_numpy(offs).cuda()
    code = {"int32": 0, "int64": 1, "float32": 2, "float64": 3, "uint32": 4, "uint64": 5}[dtype]
    lib = _lib.load()
    ps.profile_reset()
    ps.profile_enable(True)
    try:
        rc = lib.ps_sort_batch(ctypes.c_void_p(o.data_ptr()), len(lens), ctypes.c_void_p(x.data_ptr()), code, 1, None)
        torch.cuda.synchronize()
        prof = ps.profile_read()
    finally:
        ps.profile_enable(False)
    assert rc == 0
    assert prof.get("batch_front", (0, 0))[0] == 1, prof
    assert set(prof) == {"batch_front"}, "segments of at most one tile take no other launch: %s" % prof
    got = x.cpu().numpy().view(keys.dtype)
    assert got.tobytes() == reference(ora, keys, offs).tobytes()


def test_batch_front_float_specials(ps, ora):
    """Signed zeros, infinities and subnormals inside warp items and tile
    items (the order-key transform on load and its inverse on store)."""
    import torch
    specials = np.array([-0.0, 0.0, np.inf, -np.inf, 5e-324, -5e-324, 1.0, -1.0], dtype=np.float64)
    lens = np.array([8, 500, 1024, 1025, 8192, 3], dtype=np.int64)
    offs = np.zeros(len(lens) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    z = synth.splitmix64(synth.seed_for("front-specials"), int(offs[-1]))
    keys = specials[(z % np.uint64(len(specials))).astype(np.int64)]
    for dt in (np.float64, np.float32):
        k = keys.astype(dt)
        x = torch.from_numpy(k.copy()).cuda()
        ps.sort_batch(x, torch.from_numpy(offs).cuda(), "regular")
        torch.cuda.synchronize()
        assert x.cpu().numpy().tobytes() == reference(ora, k, offs).tobytes()


def test_batch_config4_shape(ps, ora):
    """Lengths log-uniform in [2^6, 2^22] (the batched benchmark's shape), 64
    segments, int32 and float32, uniform and few-unique keys."""
    import torch
    for dtype, dist in (("int32", "uniform"), ("float32", "few_unique")):
        z = synth.splitmix64(11, 64)
        u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        lens = np.floor(2.0 ** (6 + 16 * u)).astype(np.int64)
        offs = np.zeros(65, dtype=np.int64)
        offs[1:] = np.cumsum(lens)
        keys = synth.keys(int(offs[-1]), dtype, dist, seed=12)
        x = to_dev(keys)
        ps.sort_batch(x, torch.from_numpy(offs).cuda(), "exact")
        torch.cuda.synchronize()
        assert x.cpu().numpy().tobytes() == reference(ora, keys, offs).tobytes()


def test_batch_argument_errors(ps):
    import ctypes
    import torch
    from paper_2305_05245_gb300 import _lib
    lib = _lib.load()
    x = torch.zeros(10, dtype=torch.int32, device="cuda")
    bad = torch.tensor([0, 5, 3, 10], dtype=torch.int64, device="cuda")  # decreasing
    assert lib.ps_sort_batch(ctypes.c_void_p(bad.data_ptr()), 3, ctypes.c_void_p(x.data_ptr()), 0, 1, None) == -1
    assert lib.ps_sort_batch(None, 0, None, 0, 1, None) == 0
    assert lib.ps_sort_batch(ctypes.c_void_p(bad.data_ptr()), 3, ctypes.c_void_p(x.data_ptr()), 9, 1, None) == -2


@pytest.mark.parametrize("dtype", ["int32", "float64"])
def test_batch_plan_run_and_cuda_graph(ps, ora, dtype):
    """A planned batch (ps_batch_plan_create / ps_batch_run) sorts like
    ps_sort_batch, and the run can be captured in a CUDA graph and replayed on
    new keys in the same buffer."""
    import torch
    keys, offs = make_batch(500, 18, dtype, "uniform", seed=synth.seed_for("plan", dtype) % 100000,
                            special=SPECIAL)
    plan = ps.BatchPlan(offs, getattr(torch, dtype), "exact")
    try:
        x = to_dev(keys)
        plan.run(x)
        torch.cuda.synchronize()
        assert x.cpu().numpy().tobytes() == reference(ora, keys, offs).tobytes()
        # capture one run, then replay it on two fresh inputs
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            x.copy_(to_dev(keys))
            plan.run(x)  # warm-up on the capture stream
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.run(x)
        for rep in range(2):
            fresh = synth.keys(len(keys), dtype, "few_unique" if rep else "uniform",
                               seed=synth.seed_for("plan-replay", dtype, rep))
            x.copy_(to_dev(fresh))
            g.replay()
            torch.cuda.synchronize()
            assert x.cpu().numpy().tobytes() == reference(ora, fresh, offs).tobytes()
    finally:
        plan.close()


@pytest.mark.parametrize("dtype,items,threads", [("int32", 16, 512), ("int64", 32, 512), ("float64", 16, 128)])
def test_batch_bins_with_tuned_launch_shapes(ps, ora, dtype, items, threads):
    """Batched size bins whose tuned entries carry a launch shape run with it,
    through ps_sort_batch and through a batch plan (whose workspace is sized
    for that shape), and every segment still equals the oracle's result."""
    import torch
    bins = range(14, 21)
    try:
        for b in bins:
            ps.autotune_set(dtype, b, 4, 4, batched=True, items_per_thread=items, block_threads=threads)
        assert all(ps.autotune_table(dtype, batched=True)[b][2:] == (items, threads) for b in bins)
        keys, offs = make_batch(300, 19, dtype, "uniform", seed=synth.seed_for("batch-shape", dtype) % 100000,
                                special=SPECIAL)
        want = reference(ora, keys, offs).tobytes()
        x = to_dev(keys)
        ps.sort_batch(x, torch.from_numpy(offs).cuda(), "exact")
        torch.cuda.synchronize()
        assert x.cpu().numpy().tobytes() == want
        plan = ps.BatchPlan(offs, getattr(torch, dtype), "regular")
        try:
            x = to_dev(keys)
            plan.run(x)
            torch.cuda.synchronize()
            assert x.cpu().numpy().tobytes() == want
        finally:
            plan.close()
    finally:
        for b in bins:
            ps.autotune_set(dtype, b, 0, 0, batched=True)
    assert ps.autotune_table(dtype, batched=True) == {}

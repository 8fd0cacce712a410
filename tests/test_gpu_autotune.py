"""The autotuner on the GPU: it fills the tuned table for every requested
size, automatic parameters then use the entries, and sorts stay exact."""
from __future__ import annotations

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


def _clear(ps, dtype, batched):
    for b in ps.autotune_table(dtype, batched):
        ps.autotune_set(dtype, b, 0, 0, batched)


def test_autotune_single(ps, ora):
    import torch
    try:
        table = ps.autotune("int32", "exact", 1 << 16, 1 << 18)
        assert sorted(table) == [16, 17, 18]
        for b, (nb, np_, it, th) in table.items():
            assert 1 <= nb <= 4096 and 1 <= np_ <= 1024
            assert (it, th) == (0, 0) or (it in (16, 32) and th in (128, 256, 512))
        n = (1 << 17) + 123
        assert ps.resolve_params(n, 0) == table[17][:2]
        x = synth.keys_torch(n, "int32", "uniform", seed=synth.seed_for("tune-single"))
        want = ora.reference_sort(x.cpu().numpy())
        ps.sort(x, "exact")
        ps.sort(x, "regular")  # sorting sorted keys again is a no-op
        torch.cuda.synchronize()
        assert x.cpu().numpy().tobytes() == want.tobytes()
    finally:
        _clear(ps, "int32", False)
    assert ps.autotune_table("int32") == {}


def test_autotune_batched(ps, ora):
    import numpy as np
    import torch
    try:
        table = ps.autotune("int64", "exact", 1 << 15, 1 << 16, batched=True)
        assert sorted(table) == [15, 16]
        assert ps.autotune_table("int64") == {}  # the single-sort table is separate
        lens = [40_000, 50_000, 20_000, 5, 70_000, 0, 33_333]
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        x = synth.keys_torch(int(offs[-1]), "int64", "few_unique", seed=synth.seed_for("tune-batch"))
        host = x.cpu().numpy()
        want = np.concatenate([ora.reference_sort(host[offs[i]:offs[i + 1]]) for i in range(len(lens))])
        ps.sort_batch(x, torch.from_numpy(offs).cuda(), "exact")
        torch.cuda.synchronize()
        assert x.cpu().numpy().tobytes() == want.tobytes()
    finally:
        _clear(ps, "int64", True)

"""A seeded random sweep of the configuration space against the oracle:
size (2 to about 3 million keys), key type, distribution, n_B, n_P (1 to
512 each, so n_B > N and n_P > N occur), pivot mode, launch shape and
records.  Each case compares the output and every intermediate (pivots,
c_k, split table, offsets) element by element.  The cases are drawn once
from a fixed seed, so a failure names a reproducible configuration."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from test_gpu_parity import assert_parity, run_gpu

pytestmark = pytest.mark.gpu

DTYPES = ["int32", "int64", "float32", "float64", "uint32", "uint64", "records"]
DISTS = ["uniform", "few_unique", "sorted", "reverse", "almost_sorted", "three_valued", "gaussian"]
SHAPES = [(0, 0), (16, 128), (16, 256), (16, 512), (32, 128), (32, 256), (32, 512)]


def _cases(count=120):
    z = synth.splitmix64(synth.seed_for("random-sweep"), 8 * count)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    out = []
    for i in range(count):
        v = u[8 * i: 8 * i + 8]
        n = int(2.0 ** (1.0 + 20.5 * v[0]))
        dtype = DTYPES[int(v[1] * len(DTYPES))]
        dist = DISTS[int(v[2] * len(DISTS))]
        if dist == "gaussian" and not dtype.startswith("float"):
            dist = "uniform"
        if dtype == "records" and dist not in ("uniform", "few_unique", "sorted"):
            dist = "few_unique"
        n_B = max(1, int(2.0 ** (9.0 * v[3])))
        n_P = max(1, int(2.0 ** (9.0 * v[4])))
        mode = "exact" if v[5] < 0.5 else "regular"
        shape = SHAPES[int(v[6] * len(SHAPES))]
        if dtype in ("uint32", "uint64", "records"):
            shape = (0, 0)  # offered through the automatic shape only here
        out.append((i, n, dtype, dist, n_B, n_P, mode, shape))
    return out


@pytest.fixture(scope="module")
def ps():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_05245_gb300 as ps
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ps


def _run_shape(ps, keys, mode, n_B, n_P, items, threads):
    import torch
    x = torch.from_numpy(keys.copy()).cuda()
    tr = ps.sort(x, mode, n_blocks=n_B, n_parts=n_P, trace=True, items_per_thread=items, block_threads=threads)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    t = {"pivots": tr.pivots.cpu().numpy().view(keys.dtype)[: max(n_P - 1, 0)], "pivot_payload": None,
         "c": tr.c.cpu().numpy()[: max(n_P - 1, 0)], "splits": tr.splits.cpu().numpy(),
         "offsets": tr.offsets.cpu().numpy()}
    return out, t


@pytest.mark.parametrize("case", _cases(), ids=lambda c: "%d-%d-%s-%s-B%d-P%d-%s-%dx%d" % (
    c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7][0], c[7][1]))
def test_random_configuration(ps, ora, case):
    i, n, dtype, dist, n_B, n_P, mode, (items, threads) = case
    seed = synth.seed_for("random-sweep-keys", i)
    if dtype == "records":
        k, p = synth.records(n, seed=seed, dist=dist)
        out, pay, t = run_gpu(ps, k, mode, n_B, n_P, payload=p)
        assert_parity(ora, k, mode, n_B, n_P, out, pay, t, payload=p)
        return
    keys = synth.keys(n, dtype, dist, seed=seed)
    if items:
        out, t = _run_shape(ps, keys, mode, n_B, n_P, items, threads)
        assert_parity(ora, keys, mode, n_B, n_P, out, None, t)
    else:
        out, pay, t = run_gpu(ps, keys, mode, n_B, n_P)
        assert_parity(ora, keys, mode, n_B, n_P, out, pay, t)

"""GPU checks at the benchmark configurations' full sizes, where the
step-by-step oracle is too slow for every case: the output must equal the
input's sorted permutation (torch.sort of the order keys canonicalises the
multiset), and the trace must satisfy the paper's definitions -- exact
splitting pivots at ranks floor(k*N/n_P) with Eq. 1 and Eq. 2, the greedy
split table, offsets as the scan of partition sizes, and regular-sampling
pivots taken from the block samples.  One 2^26 case is also compared with
the full oracle element by element."""
from __future__ import annotations

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

_INPUTS = {}


@pytest.fixture(scope="module")
def ps():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_05245_gb300 as ps
    assert torch.cuda.is_available()
    return ps


def order_key(t):
    """int tensor whose signed order is the sort order of t (bijective)."""
    import torch
    if t.dtype == torch.float32:
        b = t.view(torch.int32)
        return b ^ ((b >> 31) & 0x7FFFFFFF)
    if t.dtype == torch.float64:
        b = t.view(torch.int64)
        return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFF)
    return t


def get_input(n, dtype, dist):
    key = (n, dtype, dist)
    if key not in _INPUTS:
        _INPUTS.clear()
        _INPUTS[key] = synth.keys_torch(n, dtype, dist, seed=synth.seed_for("full", n, dtype, dist))
    return _INPUTS[key]


def check_sort_and_trace(ps, x0, mode, n_B, n_P):
    import torch
    x = x0.clone()
    tr = ps.sort(x, mode, n_blocks=n_B, n_parts=n_P, trace=True)
    torch.cuda.synchronize()
    N = x.numel()
    ok_in, ok_out = order_key(x0), order_key(x)
    ref = torch.sort(ok_in)[0]
    assert torch.equal(ref, ok_out), "output is not the sorted permutation of the input"
    L = -(-N // n_B)
    off = tr.offsets
    s = tr.splits
    assert int(off[0]) == 0 and int(off[-1]) == N
    assert torch.equal(off, s.sum(dim=0)), "offsets are not the column sums of the split table"
    piv = order_key(tr.pivots[: n_P - 1])
    k = torch.arange(1, n_P, device=x.device, dtype=torch.int64)
    if mode == "exact":
        rk = (k * N) // n_P
        assert torch.equal(off[1:-1], rk), "exact splitting must give partitions of floor(k*N/n_P)"
        want = ref[torch.clamp(rk - 1, min=0)]
        assert torch.equal(piv, want), "P_k is not the element of rank r_k (Eq. 1)"
        below = torch.searchsorted(ref, piv, right=False)
        assert torch.equal(tr.c[: n_P - 1], rk - below), "c_k differs from Eq. 2"
    if N % n_B == 0:
        blocks = torch.sort(ok_in.view(n_B, L), dim=1)[0]
        pv = piv.unsqueeze(0).expand(n_B, -1).contiguous()
        lb = torch.searchsorted(blocks, pv, right=False)
        ub = torch.searchsorted(blocks, pv, right=True)
        if mode == "exact":
            eq = ub - lb
            before = torch.cumsum(eq, dim=0) - eq
            take = torch.minimum(eq, torch.clamp(tr.c[: n_P - 1].unsqueeze(0) - before, min=0))
            assert torch.equal(s[:, 1:-1], lb + take), "split table differs from the greedy tie fill"
        else:
            assert torch.equal(s[:, 1:-1], ub), "regular-sampling splits are not #{x <= P_k}"
            j = torch.arange(1, n_P, device=x.device, dtype=torch.int64)
            samples = blocks[:, (j * L) // n_P].reshape(-1)
            pool = torch.sort(samples)[0]
            q = (k - 1) * n_B + (n_B - 1) // 2
            assert torch.equal(piv, pool[q]), "regular-sampling pivots differ from the sample pool"


PAIRS = [(128, 2048), (512, 512), (2048, 128)]
CFG2 = [(d, t) for d in ("int32", "int64", "float32", "float64")
        for t in ("uniform", "sorted", "reverse", "few_unique")] + [("float64", "gaussian")]


@pytest.mark.parametrize("dtype,dist", CFG2)
@pytest.mark.parametrize("mode", ["regular", "exact"])
def test_config_2p26(ps, dtype, dist, mode):
    """N = 2^26 across dtypes and distributions, both pivot modes, three of the
    (n_B, n_P) pairs of {128, 512, 2048}^2."""
    x0 = get_input(1 << 26, dtype, dist)
    for n_B, n_P in PAIRS:
        check_sort_and_trace(ps, x0, mode, n_B, n_P)


@pytest.mark.parametrize("mode", ["regular", "exact"])
def test_config_2p26_all_pairs(ps, mode):
    x0 = get_input(1 << 26, "int32", "uniform")
    for n_B in (128, 512, 2048):
        for n_P in (128, 512, 2048):
            check_sort_and_trace(ps, x0, mode, n_B, n_P)


def test_config_2p26_oracle_elementwise(ps, ora):
    """One full-size case against the step-by-step oracle, element by element."""
    import torch
    keys = synth.keys(1 << 26, "int64", "uniform", seed=synth.seed_for("full-oracle"))
    x = torch.from_numpy(keys.copy()).cuda()
    tr = ps.sort(x, "exact", n_blocks=512, n_parts=512, trace=True)
    torch.cuda.synchronize()
    ref = ora.sort(keys, 1, 512, 512)
    assert np.array_equal(x.cpu().numpy(), ref.out)
    assert np.array_equal(tr.splits.cpu().numpy(), ref.splits)
    assert np.array_equal(tr.pivots.cpu().numpy()[:511], ref.pivots)
    assert np.array_equal(tr.c.cpu().numpy()[:511], ref.c)


@pytest.mark.parametrize("dtype,dist,n_B,n_P", [("int64", "uniform", 0, 0), ("int64", "uniform", 128, 128),
                                                ("float64", "gaussian", 0, 0)])
def test_config_2p30(ps, dtype, dist, n_B, n_P):
    """N = 2^30, exact splitting, in the launch configuration bench.py times."""
    x0 = get_input(1 << 30, dtype, dist)
    nb, np_ = ps.resolve_params(1 << 30, 1 if dtype == "int64" else 3, n_B, n_P)
    check_sort_and_trace(ps, x0, "exact", nb, np_)


def test_records_2p28(ps):
    """2^28 records (uint64 uniform key, uint32 payload = index), exact
    splitting: ordered by (key, payload); pivots are the records of rank r_k."""
    import torch
    n = 1 << 28
    k0 = synth.keys_torch(n, "uint64", "uniform", seed=synth.seed_for("rec28"))
    p0 = torch.arange(n, dtype=torch.int64, device=k0.device).to(torch.int32)
    k, p = k0.clone(), p0.clone()
    tr = ps.sort_pairs(k, p, "exact", trace=True)
    torch.cuda.synchronize()
    # unsigned 64-bit key order as signed order, then payload (= index, distinct)
    sk = k0 ^ (-(1 << 63))
    order = torch.sort(p0.to(torch.int64) & 0xFFFFFFFF, stable=True)[1]
    order = order[torch.sort(sk[order], stable=True)[1]]
    assert torch.equal(k, k0[order]) and torch.equal(p, p0[order])
    N, n_P = n, tr.n_parts
    kk = torch.arange(1, n_P, device=k.device, dtype=torch.int64)
    rk = (kk * N) // n_P
    assert torch.equal(tr.offsets[1:-1], rk)
    assert torch.equal(tr.pivots[: n_P - 1], k[rk - 1]) and torch.equal(tr.pivot_payload[: n_P - 1], p[rk - 1])


def _multiset_hash(t):
    """Order-independent 64-bit hash of a tensor's values (sum of SplitMix64
    finalisers of the bit patterns, wrapping), in chunks."""
    import torch
    acc = torch.zeros((), dtype=torch.int64, device=t.device)
    bits = t.view(torch.int32) if t.element_size() == 4 else t.view(torch.int64)
    for lo in range(0, t.numel(), 1 << 27):
        z = bits[lo:lo + (1 << 27)].to(torch.int64)
        acc = acc + synth._mix_t(z * -7046029254386353131 + 1).sum()
    return int(acc)


@pytest.mark.parametrize("dtype", ["int32", "int64"])
def test_beyond_2p31_keys(ps, dtype):
    """N = 2^31 + 12,345 keys (element indices beyond 32 bits), exact splitting
    with automatic parameters: non-decreasing, the same multiset, and the
    partition offsets of Eq. 1."""
    import torch
    n = (1 << 31) + 12_345
    _INPUTS.clear()
    torch.cuda.empty_cache()
    x = synth.keys_torch(n, dtype, "uniform", seed=synth.seed_for("2p31", dtype))
    h0 = _multiset_hash(x)
    code = 0 if dtype == "int32" else 1
    nb, np_ = ps.resolve_params(n, code)
    tr = ps.sort(x, "exact", n_blocks=nb, n_parts=np_, trace=True)
    torch.cuda.synchronize()
    ok = True
    for lo in range(0, n - 1, 1 << 28):
        seg = x[lo:min(n, lo + (1 << 28) + 1)]
        ok = ok and bool((seg[1:] >= seg[:-1]).all())
    assert ok, "output is not non-decreasing"
    assert _multiset_hash(x) == h0, "output is not a permutation of the input"
    k = torch.arange(1, np_, device=x.device, dtype=torch.int64)
    assert torch.equal(tr.offsets[1:-1], (k * n) // np_)
    assert int(tr.offsets[-1]) == n
    del x, tr
    torch.cuda.empty_cache()

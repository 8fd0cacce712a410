"""The paper's remaining Table 1 inputs on the GPU: AlmostSorted and
Duplicate3 (uint32), Pair (16-byte key + index records) and Particle (96-byte
key + particle data records, sorted by the uint64 key), against the oracle;
and the PSRS imbalance on Duplicate3 that Sec. 2.3 and Sec. 4 describe."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from test_gpu_parity import MODES, assert_parity, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_05245_gb300 as ps
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ps


@pytest.mark.parametrize("mode", ["regular", "exact"])
@pytest.mark.parametrize("dist", ["almost_sorted", "three_valued"])
@pytest.mark.parametrize("n", [1_000_003, 48 * 1000])
def test_almost_sorted_and_duplicate3(ps, ora, n, dist, mode):
    """uint32 keys, n_B = n_P = 48 (the paper runs one block and one partition
    per thread on 48 cores): output and every intermediate equal the oracle's."""
    keys = synth.keys(n, "uint32", dist, seed=synth.seed_for("table1", n, dist))
    out, pay, t = run_gpu(ps, keys, mode, 48, 48)
    assert_parity(ora, keys, mode, 48, 48, out, pay, t)


def test_duplicate3_partition_balance(ps, ora):
    """Three distinct values: regular sampling leaves at most three non-empty
    partitions (one holds at least N/3 keys), exact splitting gives every
    partition floor or ceil of N/n_P (Eq. 1, Eq. 2)."""
    n, parts = 2_000_000, 48
    keys = synth.keys(n, "uint32", "three_valued", seed=synth.seed_for("dup3-balance"))
    sizes = {}
    for mode in ("regular", "exact"):
        out, pay, t = run_gpu(ps, keys, mode, parts, parts)
        assert_parity(ora, keys, mode, parts, parts, out, pay, t)
        sizes[mode] = np.diff(t["offsets"])
    assert np.count_nonzero(sizes["regular"]) <= 3
    assert sizes["regular"].max() >= n // 3
    assert sizes["exact"].min() >= n // parts and sizes["exact"].max() <= -(-n // parts)


def _records(n, words, key_word, key_dist, seed):
    """n records of `words` 64-bit words: the key (uint64) at key_word, the
    record's index in the word after it (Pair) and seeded data elsewhere."""
    rec = synth.keys(n * words, "uint64", "uniform", seed=seed).reshape(n, words)
    rec[:, key_word] = synth.keys(n, "uint64", key_dist, seed=seed ^ 0x77)
    if words > 1:
        rec[:, (key_word + 1) % words] = np.arange(n, dtype=np.uint64)
    return rec


def _expected(ora, rec, key_word, mode, n_B, n_P):
    """The four steps on (key, input position) in the oracle, then the
    records in that order."""
    n = rec.shape[0]
    r = ora.sort(rec[:, key_word].copy(), MODES[mode], n_B, n_P, payload=np.arange(n, dtype=np.uint32))
    return rec[r.out_payload.astype(np.int64)]


def _gpu_struct(ps, rec, key_word, mode, n_B, n_P):
    import torch
    x = torch.from_numpy(rec.view(np.int64).copy()).cuda()
    ps.sort_struct(x, key_offset=8 * key_word, pivot_mode=mode, n_blocks=n_B, n_parts=n_P)
    torch.cuda.synchronize()
    return x.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("mode", ["regular", "exact"])
@pytest.mark.parametrize("name,n,words,key_word,key_dist,n_B,n_P", [
    ("pair", 1_000_003, 2, 0, "uniform", 48, 48),
    ("pair-ties", 200_001, 2, 0, "few_unique", 16, 12),
    ("particle", 300_007, 12, 0, "uniform", 48, 48),
    ("key-inside", 100_003, 3, 1, "uniform", 7, 5),
    ("key-last", 65_537, 5, 4, "three_valued", 4, 4),
    ("one-word", 10_007, 1, 0, "few_unique", 3, 2),
    ("tiny", 3, 12, 0, "uniform", 1, 1),
])
def test_struct_records(ps, ora, name, n, words, key_word, key_dist, n_B, n_P, mode):
    """ps_sort_struct equals the oracle's (key, position) order applied to the
    records, bit for bit (equal keys keep their input order)."""
    rec = _records(n, words, key_word, key_dist, synth.seed_for("struct", name))
    got = _gpu_struct(ps, rec, key_word, mode, n_B, n_P)
    want = _expected(ora, rec, key_word, mode, n_B, n_P)
    assert np.array_equal(got, want), "%s: %d records differ" % (name, int((got != want).any(axis=1).sum()))


@pytest.mark.parametrize("name,n,words", [("pair", 100_000_000, 2), ("particle", 20_000_000, 12)])
def test_struct_full_size(ps, name, n, words):
    """Table 1 sizes (N = 10^8 Pair; 2*10^7 Particle, 1.9 GB) with automatic
    parameters, checked on the device: keys non-decreasing, equal keys in
    input order, and every row equal to the input row it came from."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(7)
    rec = torch.randint(-(1 << 62), 1 << 62, (n, words), dtype=torch.int64, device="cuda", generator=g)
    rec[:, 0] = synth.splitmix64_torch(synth.seed_for("struct-full", name), n)
    if words > 1:
        rec[:, 1] = torch.arange(n, device="cuda")
    orig = rec.clone()
    ps.sort_struct(rec, pivot_mode="exact")
    torch.cuda.synchronize()
    k = rec[:, 0] ^ (-(1 << 63))  # unsigned order as signed
    assert bool((k[1:] >= k[:-1]).all())
    ties = k[1:] == k[:-1]
    assert bool((rec[1:, 1][ties] > rec[:-1, 1][ties]).all())
    assert torch.equal(orig[rec[:, 1]], rec)

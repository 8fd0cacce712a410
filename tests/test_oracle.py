"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the worked
examples printed in the paper (Fig. 1, Fig. 2), brute-force insertion sort on
every tiny input, the closed form of exact-splitting pivots (Eq. 1, Eq. 2),
the partition definition P_k < x <= P_{k+1} (Sec. 2), and Python's own float
and tuple ordering.
"""
from __future__ import annotations

import itertools
import math
import struct

import numpy as np
import pytest

import synth
from _helpers import (float_total_key, insertion_sort, is_nondecreasing_total,
                      multiset_hash, read_golden)

MODES = {"regular": 0, "exact": 1}


@pytest.mark.parametrize("name", ["fig1_regular.txt", "fig2a_regular.txt", "fig2b_exact.txt"])
def test_worked_examples(ora, name):
    g = read_golden(name)
    r = ora.sort(g["input"], MODES[g["mode"]], g["n_blocks"], g["n_parts"])
    np.testing.assert_array_equal(r.out, g["output"])
    np.testing.assert_array_equal(r.pivots, g["pivots"])
    np.testing.assert_array_equal(r.splits, g["splits"])
    np.testing.assert_array_equal(r.offsets, g["offsets"])
    if "c" in g:
        np.testing.assert_array_equal(r.c, g["c"])


def _check_partition_invariants(keys, r, mode, n_B, n_P):
    """Checks that follow from the paper's definitions alone."""
    N = len(keys)
    s = r.splits
    L = -(-N // n_B) if N else 0
    srt = sorted(keys.tolist())
    # split rows are monotone and span each block
    for b in range(n_B):
        m = max(0, min((b + 1) * L, N) - min(b * L, N))
        assert s[b, 0] == 0 and s[b, n_P] == m
        assert np.all(np.diff(s[b]) >= 0)
    # offsets are the exclusive scan of partition totals (Sec. 2)
    tot = (s[:, 1:] - s[:, :-1]).sum(axis=0)
    assert r.offsets[0] == 0 and np.array_equal(np.diff(r.offsets), tot)
    # partition k of the output holds global ranks [O_k, O_{k+1})
    out = r.out.tolist()
    assert out == srt
    if N == 0:
        return
    if mode == 1:
        for k in range(1, n_P):
            rk = (k * N) // n_P
            pk = srt[rk - 1] if rk >= 1 else srt[0]
            assert r.pivots[k - 1] == pk                     # closed form of Eq. 1 (smallest P_k)
            below = sum(1 for x in srt if x < pk)
            le = sum(1 for x in srt if x <= pk)
            assert below <= rk <= le                         # Eq. 1
            assert r.c[k - 1] == rk - below                  # Eq. 2
            assert r.offsets[k] == rk                        # equal partition sizes
        sizes = np.diff(r.offsets)
        assert sizes.min() >= N // n_P and sizes.max() <= -(-N // n_P)
    else:
        piv = r.pivots.tolist()
        for k in range(n_P):
            seg = out[r.offsets[k]:r.offsets[k + 1]]
            lo = piv[k - 1] if k >= 1 else None
            hi = piv[k] if k < n_P - 1 else None
            for x in seg:                                    # P_k < x <= P_{k+1} (Sec. 2)
                assert lo is None or x > lo
                assert hi is None or x <= hi


@pytest.mark.parametrize("n_B,n_P", [(1, 1), (2, 2), (3, 2), (2, 3), (4, 4), (8, 3), (3, 8)])
@pytest.mark.parametrize("mode", [0, 1])
def test_bruteforce_exhaustive_tiny(ora, n_B, n_P, mode):
    """Every input of length <= 7 over a 3-value alphabet (plus the worst case
    of all-equal runs) against insertion sort and the paper's definitions."""
    for n in range(0, 8):
        for tup in itertools.product((-1, 0, 7), repeat=n):
            keys = np.array(tup, dtype=np.int32)
            r = ora.sort(keys, mode, n_B, n_P)
            assert r.out.tolist() == insertion_sort(tup)
            _check_partition_invariants(keys, r, mode, n_B, n_P)


@pytest.mark.parametrize("dtype", ["int32", "int64", "uint32", "uint64"])
@pytest.mark.parametrize("mode", [0, 1])
def test_random_small_ints(ora, dtype, mode):
    for rep in range(40):
        n = int(synth.splitmix64(rep, 1)[0] % 65)
        a = synth.keys(n, dtype, "uniform", seed=synth.seed_for("small", dtype, rep))
        n_B = 1 + rep % 7
        n_P = 1 + (rep * 5) % 9
        r = ora.sort(a, mode, n_B, n_P)
        assert r.out.tolist() == insertion_sort(a.tolist())
        _check_partition_invariants(a, r, mode, n_B, n_P)


SPECIAL_F32 = [0.0, -0.0, 1.0, -1.0, float("inf"), float("-inf"), 3.4028234663852886e38,
               -3.4028234663852886e38, 1e-45, -1e-45, 1.17549435e-38, -1.17549435e-38, 0.5]
SPECIAL_F64 = [0.0, -0.0, 1.0, -1.0, float("inf"), float("-inf"), 1.7976931348623157e308,
               -1.7976931348623157e308, 5e-324, -5e-324, 2.2250738585072014e-308, 0.1, -0.1]


@pytest.mark.parametrize("dtype,special", [("float32", SPECIAL_F32), ("float64", SPECIAL_F64)])
@pytest.mark.parametrize("mode", [0, 1])
def test_float_total_order(ora, dtype, special, mode):
    """-0.0 < +0.0, denormals, infinities and the extreme finite values sort by
    Python's float order (ties of +-0 broken by the sign)."""
    dt = np.float32 if dtype == "float32" else np.float64
    rng_keys = synth.keys(200, dtype, "gaussian", seed=5)
    for rep in range(20):
        perm = synth.splitmix64(rep, len(special) * 3) % np.uint64(len(special))
        a = np.concatenate([np.array([special[int(i)] for i in perm], dtype=dt),
                            rng_keys[: 10 * rep]])
        r = ora.sort(a, mode, 1 + rep % 5, 1 + rep % 6)
        want = insertion_sort(a.tolist(), key=float_total_key)
        got = r.out.tolist()
        assert [struct.pack("<d", x) for x in got] == [struct.pack("<d", x) for x in want]


def check_float_pivots(ora, lib=None):
    """Exact-splitting pivots of float keys, bit for bit.  By Eq. 1 (reading:
    the smallest admissible value) P_k is the element of rank r_k = floor(k N /
    n_P) of the input in IEEE total order; the reference order comes from
    Python's float comparison (float_total_key), and pivots are compared as
    packed bytes so that -0.0 and +0.0, or two NaN-free values with equal
    magnitude, cannot be confused.  n_P = N makes every element but the last a
    pivot, so each special value (signed zeros, infinities, denormals, extreme
    finite values, negatives) is returned as a pivot at least once."""
    for dtype, special, fmt in (("float32", SPECIAL_F32, "<f"), ("float64", SPECIAL_F64, "<d")):
        dt = np.float32 if dtype == "float32" else np.float64
        neg = -np.abs(synth.keys(12, dtype, "gaussian", seed=41))
        for rep in range(10):
            perm = synth.splitmix64(rep + 500, 2 * len(special)) % np.uint64(len(special))
            a = np.concatenate([np.array([special[int(i)] for i in perm], dtype=dt), neg[: rep + 2]])
            N = len(a)
            want = insertion_sort(a.tolist(), key=float_total_key)
            for n_B, n_P in ((1 + rep % 4, N), (2 + rep % 3, 2 + rep % 7)):
                r = ora.sort(a, 1, n_B, n_P, lib=lib)
                for k in range(1, n_P):
                    rk = (k * N) // n_P
                    pk = want[rk - 1] if rk >= 1 else want[0]
                    assert struct.pack(fmt, float(r.pivots[k - 1])) == struct.pack(fmt, pk), \
                        "%s pivot %d of %d: got %r, want %r" % (dtype, k, n_P, float(r.pivots[k - 1]), pk)


def test_float_pivots_bit_exact(ora):
    check_float_pivots(ora)


def test_int_extremes(ora):
    a = np.array([2**31 - 1, -2**31, 0, -1, 1, -2**31, 2**31 - 1, 5], dtype=np.int32)
    for mode in (0, 1):
        assert ora.sort(a, mode, 3, 3).out.tolist() == sorted(a.tolist())
    b = np.array([2**63 - 1, -2**63, 0, -1, 1, -2**63, 12], dtype=np.int64)
    for mode in (0, 1):
        assert ora.sort(b, mode, 2, 4).out.tolist() == sorted(b.tolist())


@pytest.mark.parametrize("mode", [0, 1])
def test_records_key_then_payload(ora, mode):
    """Records order by (key, payload): compared with Python's tuple order."""
    for rep in range(30):
        n = 1 + rep * 3
        k = synth.keys(n, "uint64", "few_unique", seed=rep) if rep % 2 else \
            synth.keys(n, "uint64", "uniform", seed=rep)
        p = (synth.splitmix64(rep + 99, n) >> np.uint64(32)).astype(np.uint32)
        r = ora.sort(k, mode, 1 + rep % 4, 1 + rep % 5, payload=p)
        want = sorted(zip(k.tolist(), p.tolist()))
        assert list(zip(r.out.tolist(), r.out_payload.tolist())) == want
        if mode == 1:
            # exact-splitting pivots are the order statistics of the records
            N, n_P = n, 1 + rep % 5
            for kk in range(1, n_P):
                rk = (kk * N) // n_P
                pk = want[rk - 1] if rk >= 1 else want[0]
                assert (int(r.pivots[kk - 1]), int(r.pivot_payload[kk - 1])) == pk


@pytest.mark.parametrize("dist", ["uniform", "few_unique", "sorted", "reverse", "three_valued"])
@pytest.mark.parametrize("mode", [0, 1])
def test_medium_invariants(ora, dist, mode):
    """N = 20000: sorted, same multiset, and the partition invariants."""
    a = synth.keys(20000, "int32", dist, seed=synth.seed_for("medium", dist))
    r = ora.sort(a, mode, 16, 12)
    assert is_nondecreasing_total(r.out)
    assert multiset_hash(r.out) == multiset_hash(a)
    assert np.array_equal(r.out, np.sort(a, kind="stable"))
    _check_partition_invariants(a, r, mode, 16, 12)


def test_pses_balance_with_few_distinct(ora):
    """Sec. 2.3: exact splitting equalises partition sizes however few distinct
    values there are; regular sampling cannot (Fig. 2(a))."""
    a = synth.keys(6000, "int32", "three_valued", seed=3)
    ex = ora.sort(a, 1, 8, 8)
    assert set(np.diff(ex.offsets).tolist()) <= {6000 // 8, -(-6000 // 8)}
    rg = ora.sort(a, 0, 8, 8)
    assert np.diff(rg.offsets).max() >= 6000 // 3     # a whole value class lands in one partition


def test_psrs_regular_sampling_bound(ora):
    """Regular sampling keeps every partition within about twice the mean for
    distinct keys (Shi & Schaeffer's PSRS bound, cited in Sec. 2.3): with n_B'
    blocks of length L, no partition exceeds 2 n_B (ceil(L/n_P) + 1)."""
    for n_B, n_P in [(4, 4), (8, 8), (16, 5), (5, 16)]:
        a = synth.keys(50000, "int64", "uniform", seed=n_B * 100 + n_P)
        r = ora.sort(a, 0, n_B, n_P)
        L = -(-50000 // n_B)
        assert np.diff(r.offsets).max() <= 2 * n_B * (-(-L // n_P) + 1)


def test_edge_shapes(ora):
    for mode in (0, 1):
        for n, n_B, n_P in [(0, 1, 1), (0, 4, 4), (1, 1, 1), (1, 3, 5), (3, 8, 2), (5, 2, 9),
                            (10, 10, 10), (7, 1, 7), (9, 9, 1)]:
            a = synth.keys(n, "int32", "uniform", seed=n * 31 + n_B)
            r = ora.sort(a, mode, n_B, n_P)
            assert r.out.tolist() == sorted(a.tolist())
            _check_partition_invariants(a, r, mode, n_B, n_P)
        a = np.full(37, 4, dtype=np.int32)
        r = ora.sort(a, mode, 5, 6)
        _check_partition_invariants(a, r, mode, 5, 6)


def test_rejects_bad_arguments(ora):
    with pytest.raises(ValueError):
        ora.sort(np.zeros(4, np.int32), 0, 0, 2)
    with pytest.raises(ValueError):
        ora.sort(np.zeros(4, np.int32), 3, 2, 2)


@pytest.mark.parametrize("dtype,dist", [("int32", "uniform"), ("int64", "few_unique"),
                                        ("float32", "gaussian"), ("float64", "gaussian"),
                                        ("uint32", "three_valued"), ("uint64", "reverse")])
def test_reference_sort_matches_oracle(ora, dtype, dist):
    """The numpy plain-definition reference agrees with the four-step oracle."""
    if dist == "gaussian" and not dtype.startswith("float"):
        pytest.skip("gaussian keys are floating point")
    a = synth.keys(30000, dtype, dist, seed=synth.seed_for("ref", dtype, dist))
    if dtype.startswith("float"):
        a[:4] = [-0.0, 0.0, -0.0, 0.0]
    got = ora.reference_sort(a)
    want = ora.sort(a, 1, 7, 9).out
    assert got.tobytes() == want.tobytes()
    k, p = synth.records(5000, seed=3, dist="few_unique")
    rk, rp = ora.reference_sort(k, p)
    r = ora.sort(k, 0, 5, 5, payload=p)
    assert np.array_equal(rk, r.out) and np.array_equal(rp, r.out_payload)

"""The oracle's pins are sharp: plant one plausible mistake at a time in a
copy of the oracle (on the CPU, in a temporary directory) and check that the
pins of test_oracle.py reject every mutant."""
from __future__ import annotations

import itertools
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from _helpers import float_total_key, insertion_sort, read_golden
from test_oracle import MODES, _check_partition_invariants, check_float_pivots

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "psort_oracle.c")

MUTANTS = {
    "psrs_pivot_upper_median": ("(nb1 - 1) / 2", "nb1 / 2"),
    "pses_no_tie_cap": ("int64_t take = eq < need ? eq : need;", "int64_t take = eq;"),
    "eq2_off_by_one": ("cc[k - 1] = r - below;", "cc[k - 1] = r - below + 1;"),
    "i32_no_sign_flip": ("case ORA_I32: return (uint64_t)((uint32_t)bits ^ 0x80000000u);",
                         "case ORA_I32: return (uint64_t)((uint32_t)bits);"),
    "f32_negatives_not_inverted": ("if (u & 0x80000000u) return (uint64_t)(uint32_t)~u;",
                                   "if (u & 0x80000000u) return (uint64_t)u;"),
    "block_length_floor": ("int64_t L = (N + n_B - 1) / n_B;", "int64_t L = N / n_B + 1;"),
    "rank_ceiling": ("int64_t r = (int64_t)(((unsigned __int128)k * (uint64_t)N) / (uint64_t)n_P);",
                     "int64_t r = (int64_t)(((unsigned __int128)k * (uint64_t)N + n_P - 1) / (uint64_t)n_P);"),
    "psrs_split_strict": ("v = count_le(blk, m, pk[k - 1], pp[k - 1]); /* x <= P_k goes below */",
                          "v = count_lt(blk, m, pk[k - 1], pp[k - 1]);"),
    "merge_takes_larger": ("if (less(&lv[b].base[lv[b].pos], &lv[a].base[lv[a].pos])) return b;",
                           "if (less(&lv[a].base[lv[a].pos], &lv[b].base[lv[b].pos])) return b;"),
    "offsets_not_scanned": ("O[k + 1] = O[k] + t;", "O[k + 1] = t;"),
    "psrs_sample_index_low": ("(unsigned __int128)j * (uint64_t)m", "(unsigned __int128)(j - 1) * (uint64_t)m"),
    "pses_rank_not_clamped": ("int64_t want = r > 0 ? r : 1;", "int64_t want = r;"),
    "pses_ties_not_counted": ("int64_t need = cc[k - 1] - taken;", "int64_t need = cc[k - 1];"),
    "pses_below_counts_equal": ("below += count_lt(a + BLO(b), BHI(b) - BLO(b), pk[k - 1], pp[k - 1]);",
                                "below += count_le(a + BLO(b), BHI(b) - BLO(b), pk[k - 1], pp[k - 1]);"),
    # the inverse order key that turns float pivots back into key bits
    "f32_pivot_branches_swapped": (
        "if (u & 0x80000000u) return (uint64_t)(u & 0x7fffffffu);\n        return (uint64_t)(uint32_t)~u;",
        "if (u & 0x80000000u) return (uint64_t)(uint32_t)~u;\n        return (uint64_t)(u & 0x7fffffffu);"),
    "f64_pivot_branches_swapped": (
        "if (k & 0x8000000000000000ull) return k & 0x7fffffffffffffffull;\n        return ~k;",
        "if (k & 0x8000000000000000ull) return ~k;\n        return k & 0x7fffffffffffffffull;"),
    "f64_pivot_negatives_sign_flip_only": (
        "if (k & 0x8000000000000000ull) return k & 0x7fffffffffffffffull;\n        return ~k;",
        "if (k & 0x8000000000000000ull) return k & 0x7fffffffffffffffull;\n        return k ^ 0x8000000000000000ull;"),
}


def _battery(ora, lib):
    """The oracle pins, run against one compiled variant."""
    for name in ["fig1_regular.txt", "fig2a_regular.txt", "fig2b_exact.txt"]:
        g = read_golden(name)
        r = ora.sort(g["input"], MODES[g["mode"]], g["n_blocks"], g["n_parts"], lib=lib)
        assert np.array_equal(r.out, g["output"])
        assert np.array_equal(r.pivots, g["pivots"])
        assert np.array_equal(r.splits, g["splits"])
        assert np.array_equal(r.offsets, g["offsets"])
        if "c" in g:
            assert np.array_equal(r.c, g["c"])
    for mode in (0, 1):
        for n_B, n_P in [(2, 2), (3, 2), (2, 3), (4, 4)]:
            for n in range(0, 6):
                for tup in itertools.product((-1, 0, 7), repeat=n):
                    keys = np.array(tup, dtype=np.int32)
                    r = ora.sort(keys, mode, n_B, n_P, lib=lib)
                    assert r.out.tolist() == insertion_sort(tup)
                    _check_partition_invariants(keys, r, mode, n_B, n_P)
        a = synth.keys(300, "float32", "gaussian", seed=4)
        a[:3] = [0.0, -0.0, -1.0]
        r = ora.sort(a, mode, 3, 4, lib=lib)
        assert r.out.tolist() == insertion_sort(a.tolist(), key=float_total_key)
    check_float_pivots(ora, lib)


def test_unmutated_passes(ora):
    _battery(ora, ora.load_library(ora.build()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_rejected(ora, tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor must occur exactly once"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(mut)])
    # each mutant runs in its own process, so a mutant that corrupts memory
    # cannot disturb the rest of the test session
    code = ("import sys; sys.path[:0] = %r; import oracle, test_oracle_mutations as m\n"
            "try:\n    m._battery(oracle, oracle.load_library(%r))\n"
            "except AssertionError:\n    sys.exit(3)\n" % ([HERE, ROOT], str(so)))
    rc = subprocess.run([sys.executable, "-c", code], capture_output=True).returncode
    assert rc == 3, "mutant %s was not rejected by the pins (rc=%d)" % (name, rc)

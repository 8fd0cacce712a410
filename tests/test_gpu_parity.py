"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element, output and every intermediate (pivots, c_k, split table,
offsets).  Sizes span many tiles and ragged tails; edge shapes included."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from _helpers import read_golden

pytestmark = pytest.mark.gpu

MODES = {"regular": 0, "exact": 1}
TORCH_DT = {}


@pytest.fixture(scope="module")
def ps():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_05245_gb300 as ps
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    TORCH_DT.update({np.dtype(np.int32): torch.int32, np.dtype(np.int64): torch.int64,
                     np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64})
    return ps


def _to_dev(a: np.ndarray):
    import torch
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32).copy()).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64).copy()).cuda()
    return torch.from_numpy(a.copy()).cuda()


def _from_dev(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def run_gpu(ps, keys: np.ndarray, mode: str, n_B: int, n_P: int, payload=None):
    """Sort on the GPU through the C ABI; return (output, payload, trace as numpy)."""
    import torch
    x = _to_dev(keys)
    if payload is None:
        code = {np.dtype(np.uint32): 4, np.dtype(np.uint64): 5}.get(keys.dtype)
        if code is None:
            tr = ps.sort(x, mode, n_blocks=n_B, n_parts=n_P, trace=True)
        else:
            tr = _sort_unsigned(ps, x, code, mode, n_B, n_P)
        torch.cuda.synchronize()
        out = _from_dev(x, keys.dtype)
        pay = None
    else:
        p = torch.from_numpy(payload.view(np.int32).copy()).cuda()
        tr = ps.sort_pairs(x, p, mode, n_blocks=n_B, n_parts=n_P, trace=True)
        torch.cuda.synchronize()
        out = _from_dev(x, np.uint64)
        pay = _from_dev(p, np.uint32)
    t = {"pivots": tr.pivots.cpu().numpy().view(keys.dtype)[: max(n_P - 1, 0)],
         "pivot_payload": tr.pivot_payload.cpu().numpy().view(np.uint32)[: max(n_P - 1, 0)],
         "c": tr.c.cpu().numpy()[: max(n_P - 1, 0)], "splits": tr.splits.cpu().numpy(),
         "offsets": tr.offsets.cpu().numpy()}
    return out, pay, t


def _sort_unsigned(ps, x, code, mode, n_B, n_P):
    """uint32/uint64 keys through ps_sort_ex with the unsigned dtype codes
    (torch tensors of the same width carry the bits)."""
    import ctypes
    from paper_2305_05245_gb300 import _lib
    lib = _lib.load()
    tr, ct = ps._make_trace(x.numel(), code, n_B, n_P, x.dtype, x.device, False)
    rc = lib.ps_sort_ex(x.data_ptr(), x.numel(), code, ps._mode(mode),
                        ctypes.byref(ps._params(n_B, n_P)), ctypes.byref(ct), ps._stream_handle(None))
    _lib.check(lib, "ps_sort_ex", rc)
    return tr


def assert_parity(ora, keys, mode, n_B, n_P, out, pay, t, payload=None, check_trace=True):
    ref = ora.sort(keys, MODES[mode], n_B, n_P, payload=payload)
    if out.tobytes() != ref.out.tobytes():
        diff = np.nonzero(out.view(np.uint8).reshape(len(out), -1) !=
                          ref.out.view(np.uint8).reshape(len(out), -1))[0]
        diff = np.unique(diff)
        raise AssertionError("output differs from the oracle at %d positions, first %s" %
                             (len(diff), diff[:5]))
    if payload is not None:
        assert np.array_equal(pay, ref.out_payload)
    if not check_trace or len(keys) < 2:
        return
    assert np.array_equal(t["splits"], ref.splits), "split table differs"
    assert np.array_equal(t["offsets"], ref.offsets), "offsets differ"
    assert t["pivots"].tobytes() == ref.pivots.tobytes(), "pivots differ"
    if payload is not None:
        assert np.array_equal(t["pivot_payload"], ref.pivot_payload)
    if mode == "exact":
        assert np.array_equal(t["c"], ref.c), "c_k differ"


@pytest.mark.parametrize("name", ["fig1_regular.txt", "fig2a_regular.txt", "fig2b_exact.txt"])
def test_worked_examples_gpu(ps, ora, name):
    g = read_golden(name)
    out, _, t = run_gpu(ps, g["input"], g["mode"], g["n_blocks"], g["n_parts"])
    np.testing.assert_array_equal(out, g["output"])
    np.testing.assert_array_equal(t["pivots"], g["pivots"])
    np.testing.assert_array_equal(t["splits"], g["splits"])
    np.testing.assert_array_equal(t["offsets"], g["offsets"])
    if "c" in g:
        np.testing.assert_array_equal(t["c"], g["c"])


@pytest.mark.parametrize("mode", ["regular", "exact"])
def test_config_small_2p20_int32(ps, ora, mode):
    """N = 2^20 int32 uniform over the full range, n_B = n_P = 64."""
    keys = synth.keys(1 << 20, "int32", "uniform", seed=synth.seed_for("cfg0", "int32", mode))
    out, pay, t = run_gpu(ps, keys, mode, 64, 64)
    assert_parity(ora, keys, mode, 64, 64, out, pay, t)


CASES = [
    # (n, dtype, dist, n_B, n_P)
    (2, "int32", "uniform", 1, 1), (3, "int64", "uniform", 2, 2), (17, "float32", "gaussian", 4, 3),
    (1000, "int32", "few_unique", 3, 7), (8191, "uint32", "uniform", 1, 4),
    (8193, "int64", "reverse", 1, 2), (16385, "float64", "gaussian", 2, 5),
    (50_001, "int32", "sorted", 7, 13), (50_001, "float32", "few_unique", 13, 7),
    (100_003, "uint64", "three_valued", 16, 16), (131_071, "int64", "almost_sorted", 5, 31),
    (300_007, "int32", "uniform", 1, 8), (300_007, "float64", "uniform", 64, 64),
    (1_000_003, "float32", "uniform", 4, 200), (1_000_003, "int64", "few_unique", 100, 3),
    (77, "int32", "uniform", 100, 9), (500, "int64", "uniform", 3, 700),
    (2_500_000, "int32", "uniform", 1, 16), (12_345, "float64", "few_unique", 4096, 2),
    # multi-level refinement of one huge group, and groups too wide to split
    # (4096 runs) that take the exact sub-chunk path
    (3_000_000, "int64", "uniform", 2, 1), (300_000, "int64", "uniform", 4096, 3),
    (1_500_000, "float32", "few_unique", 3, 2),
]


@pytest.mark.parametrize("mode", ["regular", "exact"])
@pytest.mark.parametrize("n,dtype,dist,n_B,n_P", CASES)
def test_parity_shapes(ps, ora, n, dtype, dist, n_B, n_P, mode):
    if dist == "gaussian" and not dtype.startswith("float"):
        pytest.skip("gaussian keys are floating point")
    keys = synth.keys(n, dtype, dist, seed=synth.seed_for("shape", n, dtype, dist))
    out, pay, t = run_gpu(ps, keys, mode, n_B, n_P)
    assert_parity(ora, keys, mode, n_B, n_P, out, pay, t)


@pytest.mark.parametrize("mode", ["regular", "exact"])
@pytest.mark.parametrize("n,dist,n_B,n_P", [(1000, "uniform", 3, 4), (100_003, "few_unique", 8, 8),
                                              (250_000, "uniform", 1, 64), (70_001, "sorted", 64, 5),
                                              (262_221, "few_unique", 2, 16)])
def test_parity_records(ps, ora, n, dist, n_B, n_P, mode):
    k, p = synth.records(n, seed=synth.seed_for("rec", n, dist), dist=dist)
    out, pay, t = run_gpu(ps, k, mode, n_B, n_P, payload=p)
    assert_parity(ora, k, mode, n_B, n_P, out, pay, t, payload=p)


def test_float_specials_gpu(ps, ora):
    vals = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 1e-45, -1e-45, 3.4e38, -3.4e38],
                    dtype=np.float32)
    keys = np.tile(vals, 3001)
    perm = np.argsort(synth.splitmix64(9, keys.size))
    keys = keys[perm]
    for mode in ("regular", "exact"):
        out, pay, t = run_gpu(ps, keys, mode, 5, 6)
        assert_parity(ora, keys, mode, 5, 6, out, pay, t)


def test_repeat_determinism(ps):
    """Same input, same bits, every time (shared-memory phases race-free)."""
    import torch
    keys = synth.keys(400_000, "int64", "few_unique", seed=77)
    ref = None
    for _ in range(10):
        x = _to_dev(keys)
        ps.sort(x, "exact", n_blocks=8, n_parts=8)
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        if ref is None:
            ref = got
        assert np.array_equal(got, ref)

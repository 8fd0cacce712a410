"""CPU oracle for the four-step parallel samplesort (arXiv 2305.05245, Sec. 2).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of bench.py may import this
package.  The product path (``paper_2305_05245_gb300``) never imports it, and
it imports nothing from the product.

``psort_oracle.c`` holds the arithmetic (plain, single-threaded C); this file
only compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psort_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

I32, I64, F32, F64, U32, U64, PAIR = range(7)
REGULAR, EXACT = 0, 1

_NP_DTYPE = {I32: np.int32, I64: np.int64, F32: np.float32, F64: np.float64,
             U32: np.uint32, U64: np.uint64, PAIR: np.uint64}

_lib = None


def build(force: bool = False) -> str:
    """Compile psort_oracle.c into liboracle.so beside it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """ctypes handle on a compiled oracle (the default one, or a variant a
    test compiled from a deliberately mutated copy of psort_oracle.c)."""
    lib = ctypes.CDLL(path)
    lib.ora_sort.restype = ctypes.c_int
    lib.ora_sort.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = load_library(_LIB)
    return _lib


@dataclass
class Result:
    """Output and intermediates of one oracle sort."""
    out: np.ndarray            # sorted keys (input dtype)
    out_payload: np.ndarray | None
    pivots: np.ndarray         # P_1..P_{n_P-1}, key dtype
    pivot_payload: np.ndarray  # payload half of each pivot (records; zeros otherwise)
    c: np.ndarray              # c_k of Eq. 2 (exact splitting; zeros for regular sampling)
    splits: np.ndarray         # (n_B, n_P+1) split table
    offsets: np.ndarray        # O_0..O_{n_P}


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def sort(keys: np.ndarray, mode: int, n_blocks: int, n_parts: int,
         payload: np.ndarray | None = None, dtype: int | None = None, lib=None) -> Result:
    """Run the oracle on ``keys`` (and ``payload`` for records)."""
    lib = lib if lib is not None else _load()
    keys = np.ascontiguousarray(keys)
    if dtype is None:
        if payload is not None:
            dtype = PAIR
        else:
            dtype = {np.dtype(np.int32): I32, np.dtype(np.int64): I64,
                     np.dtype(np.float32): F32, np.dtype(np.float64): F64,
                     np.dtype(np.uint32): U32, np.dtype(np.uint64): U64}[keys.dtype]
    n = keys.shape[0]
    kd = _NP_DTYPE[dtype]
    keys = keys.astype(kd, copy=False)
    pay = None
    if dtype == PAIR:
        pay = np.ascontiguousarray(payload, dtype=np.uint32)
    out = np.empty(n, dtype=kd)
    out_pay = np.empty(n, dtype=np.uint32) if dtype == PAIR else None
    npv = max(n_parts - 1, 0)
    piv_bits = np.zeros(max(npv, 1), dtype=np.uint64)
    piv_pay = np.zeros(max(npv, 1), dtype=np.uint32)
    c = np.zeros(max(npv, 1), dtype=np.int64)
    splits = np.zeros((n_blocks, n_parts + 1), dtype=np.int64)
    offsets = np.zeros(n_parts + 1, dtype=np.int64)
    rc = lib.ora_sort(dtype, mode, n, _ptr(keys), _ptr(pay), n_blocks, n_parts,
                      _ptr(out), _ptr(out_pay), _ptr(piv_bits), _ptr(piv_pay), _ptr(c),
                      _ptr(splits), _ptr(offsets))
    if rc != 0:
        raise ValueError("oracle rejected its arguments (rc=%d)" % rc)
    if kd in (np.int32, np.uint32, np.float32):
        pivots = piv_bits[:npv].astype(np.uint32).view(kd)
    else:
        pivots = piv_bits[:npv].view(kd)
    return Result(out, out_pay, pivots.copy(), piv_pay[:npv].copy(), c[:npv].copy(),
                  splits, offsets)


def order_key(keys: np.ndarray) -> np.ndarray:
    """Order key of each key as an unsigned integer (numpy restatement of the
    same reading as psort_oracle.c: sign flip for signed integers, IEEE
    totalOrder bits for floats)."""
    k = np.ascontiguousarray(keys)
    if k.dtype == np.int32:
        return k.view(np.uint32) ^ np.uint32(0x80000000)
    if k.dtype == np.int64:
        return k.view(np.uint64) ^ np.uint64(0x8000000000000000)
    if k.dtype == np.float32:
        u = k.view(np.uint32)
        neg = (u >> np.uint32(31)).astype(bool)
        return np.where(neg, ~u, u | np.uint32(0x80000000))
    if k.dtype == np.float64:
        u = k.view(np.uint64)
        neg = (u >> np.uint64(63)).astype(bool)
        return np.where(neg, ~u, u | np.uint64(0x8000000000000000))
    if k.dtype in (np.uint32, np.uint64):
        return k
    raise TypeError(k.dtype)


def reference_sort(keys: np.ndarray, payload: np.ndarray | None = None):
    """The method's final result by its plain definition: the unique
    permutation of the input that is ascending in (order key, payload).
    numpy's stable argsort is the library step; used for inputs too large
    for the step-by-step oracle."""
    ok = order_key(keys)
    if payload is None:
        return keys[np.argsort(ok, kind="stable")]
    idx = np.lexsort((np.asarray(payload, dtype=np.uint32), ok))
    return keys[idx], np.asarray(payload)[idx]

"""Small helpers shared by the test files (no sorting arithmetic here)."""
from __future__ import annotations

import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    """Parse a tests/golden/*.txt fixture: '#' comments, then 'field values'."""
    d = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            d[key] = rest.strip()
    out = {"dtype": d["dtype"], "mode": d["mode"], "n_blocks": int(d["n_blocks"]),
           "n_parts": int(d["n_parts"])}
    np_dt = {"int32": np.int32, "int64": np.int64, "float32": np.float32,
             "float64": np.float64}[d["dtype"]]
    out["input"] = np.array([float(x) if "float" in d["dtype"] else int(x)
                             for x in d["input"].split()], dtype=np_dt)
    out["output"] = np.array([float(x) if "float" in d["dtype"] else int(x)
                              for x in d["output"].split()], dtype=np_dt)
    out["pivots"] = np.array([float(x) if "float" in d["dtype"] else int(x)
                              for x in d["pivots"].split()], dtype=np_dt)
    if "c" in d:
        out["c"] = np.array([int(x) for x in d["c"].split()], dtype=np.int64)
    out["splits"] = np.array([[int(x) for x in row.split()] for row in d["splits"].split(";")],
                             dtype=np.int64)
    out["offsets"] = np.array([int(x) for x in d["offsets"].split()], dtype=np.int64)
    return out


def float_total_key(x: float):
    """Sort key for finite/inf floats where -0.0 sorts before +0.0 (IEEE
    totalOrder restricted to non-NaN values), built from Python's own float
    comparison rather than from bit patterns."""
    return (x, math.copysign(1.0, x))


def insertion_sort(seq, key=lambda v: v):
    """Textbook insertion sort (stable), used only as a brute-force reference."""
    a = list(seq)
    for i in range(1, len(a)):
        cur = a[i]
        j = i - 1
        while j >= 0 and key(a[j]) > key(cur):
            a[j + 1] = a[j]
            j -= 1
        a[j + 1] = cur
    return a


_M = np.uint64(0xFF51AFD7ED558CCD)


def multiset_hash(a: np.ndarray) -> int:
    """Order-independent 64-bit hash of the multiset of bit patterns:
    sum over elements of a mixed 64-bit image, modulo 2^64."""
    if a.dtype.itemsize == 4:
        u = a.view(np.uint32).astype(np.uint64)
    else:
        u = a.view(np.uint64)
    with np.errstate(over="ignore"):
        z = u ^ (u >> np.uint64(33))
        z = z * _M
        z = z ^ (z >> np.uint64(29))
        return int(np.sum(z, dtype=np.uint64))


def is_nondecreasing_total(a: np.ndarray) -> bool:
    """Non-decreasing in the key order (floats: -0.0 before +0.0)."""
    if a.size < 2:
        return True
    if a.dtype.kind == "f":
        x, y = a[:-1], a[1:]
        lt = x < y
        eq = x == y
        zero_ok = ~((x == 0) & (y == 0) & ~np.signbit(x) & np.signbit(y))
        return bool(np.all(lt | (eq & zero_ok)))
    return bool(np.all(a[:-1] <= a[1:]))

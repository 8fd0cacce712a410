"""Seeded synthetic inputs for the samplesort tests and benchmark.

This module holds none of the sorting method's arithmetic: it only draws
numbers.  Both the CUDA path (through tests and bench.py) and the CPU oracle
are fed from here, so neither side generates its own inputs.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): output i of a stream with seed s is
mix(s + (i + 1) * 0x9E3779B97F4A7C15), with mix the published finaliser.

Distributions follow the shapes of the paper's Table 1 workloads and the
benchmark configurations: uniform (integers over the full range, floats in
[0, 1) from 24 / 53 random mantissa bits), sorted, reverse sorted, few-unique
(16 distinct values), Gaussian (Box-Muller, mean 0, sd 1), almost sorted
(floor(sqrt(N))/2 random transpositions of 0..N-1) and three-valued
(uniform over {0, 1, 2}).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DTYPES = {"int32": np.int32, "int64": np.int64, "float32": np.float32,
          "float64": np.float64, "uint32": np.uint32, "uint64": np.uint64}
DISTS = ("uniform", "sorted", "reverse", "few_unique", "gaussian", "almost_sorted",
         "three_valued")

_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+n-1 of the SplitMix64 stream with this seed."""
    out = np.empty(n, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, n, _CHUNK):
            hi = min(n, lo + _CHUNK)
            i = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            out[lo:hi] = _mix(s + i * GAMMA)
    return out


def seed_for(*parts) -> int:
    """Derive a 64-bit seed from a tuple of labels (config, dtype, dist, rep...)."""
    h = 0x243F6A8885A308D3
    for p in parts:
        for ch in str(p).encode():
            h = int(splitmix64(h ^ ch, 1)[0])
        h = int(splitmix64(h ^ 0xFF, 1)[0])
    return h


def _uniform_bits_to(dtype, z: np.ndarray) -> np.ndarray:
    if dtype == np.int32:
        return (z >> np.uint64(32)).astype(np.uint32).view(np.int32)
    if dtype == np.uint32:
        return (z >> np.uint64(32)).astype(np.uint32)
    if dtype == np.int64:
        return z.view(np.int64)
    if dtype == np.uint64:
        return z
    if dtype == np.float32:
        return ((z >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)
    if dtype == np.float64:
        return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    raise ValueError(dtype)


def keys(n: int, dtype: str = "int32", dist: str = "uniform", seed: int = 1) -> np.ndarray:
    """n seeded keys of the given dtype name and distribution."""
    dt = DTYPES[dtype]
    if dist == "uniform":
        return _uniform_bits_to(dt, splitmix64(seed, n))
    if dist == "sorted":
        return np.sort(_uniform_bits_to(dt, splitmix64(seed, n)), kind="stable")
    if dist == "reverse":
        return np.sort(_uniform_bits_to(dt, splitmix64(seed, n)), kind="stable")[::-1].copy()
    if dist == "few_unique":
        vals = _uniform_bits_to(dt, splitmix64(seed ^ 0x5A5A5A5A, 16))
        idx = (splitmix64(seed, n) >> np.uint64(60)).astype(np.int64)
        return vals[idx]
    if dist == "gaussian":
        if dt not in (np.float32, np.float64):
            raise ValueError("gaussian keys are floating point")
        z1 = splitmix64(seed, n)
        z2 = splitmix64(seed ^ 0xC3C3C3C3C3C3C3C3, n)
        u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
        u2 = (z2 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        return g.astype(dt)
    if dist == "almost_sorted":
        a = np.arange(n, dtype=np.int64)
        n_swaps = int(np.floor(np.sqrt(n))) // 2
        if n >= 2 and n_swaps > 0:
            z = splitmix64(seed, 2 * n_swaps)
            i = (z[0::2] % np.uint64(n)).astype(np.int64)
            j = (z[1::2] % np.uint64(n)).astype(np.int64)
            for x, y in zip(i, j):
                a[x], a[y] = a[y], a[x]
        return a.astype(dt)
    if dist == "three_valued":
        z = splitmix64(seed, n)
        return (z % np.uint64(3)).astype(dt)
    raise ValueError(dist)


def records(n: int, seed: int = 1, dist: str = "uniform"):
    """(uint64 key, uint32 payload = original index) records, SoA."""
    k = keys(n, "uint64", dist, seed)
    p = np.arange(n, dtype=np.uint64).astype(np.uint32)
    return k, p


# ----------------------------------------------------------------- device twin
def _mix_t(z):
    """SplitMix64 finaliser on int64 torch tensors (two's-complement wrap;
    logical right shifts emulated with masks)."""
    import torch

    def shr(x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)

    m1 = torch.tensor(0xBF58476D1CE4E5B9 - (1 << 64), dtype=torch.int64, device=z.device)
    m2 = torch.tensor(0x94D049BB133111EB - (1 << 64), dtype=torch.int64, device=z.device)
    z = (z ^ shr(z, 30)) * m1
    z = (z ^ shr(z, 27)) * m2
    return z ^ shr(z, 31)


def splitmix64_torch(seed: int, n: int, device="cuda", start: int = 0):
    """The same stream as splitmix64(), computed on a torch device (int64
    tensor holding the uint64 bits)."""
    import torch
    s = seed & 0xFFFFFFFFFFFFFFFF
    s = s - (1 << 64) if s >= (1 << 63) else s
    g = 0x9E3779B97F4A7C15 - (1 << 64)
    out = torch.empty(n, dtype=torch.int64, device=device)
    step = 1 << 26
    for lo in range(0, n, step):
        hi = min(n, lo + step)
        i = torch.arange(start + lo + 1, start + hi + 1, dtype=torch.int64, device=device)
        out[lo:hi] = _mix_t(i * g + s)
    return out


def keys_torch(n: int, dtype: str = "int64", dist: str = "uniform", seed: int = 1, device="cuda"):
    """Device twin of keys() for the integer dtypes (bit-identical output) and
    the float uniform/few-unique cases; returns a torch tensor (uint dtypes as
    same-width signed storage)."""
    import torch
    z = splitmix64_torch(seed, n, device)
    if dist in ("uniform", "sorted", "reverse"):
        k = _uniform_bits_torch(dtype, z)
        if dist != "uniform":
            k = _sort_like_numpy(k, dtype)
            if dist == "reverse":
                k = torch.flip(k, [0])
        return k
    if dist == "few_unique":
        vals = _uniform_bits_torch(dtype, splitmix64_torch(seed ^ 0x5A5A5A5A, 16, device))
        idx = (z >> 60) & 15
        return vals[idx]
    if dist == "gaussian":
        # Box-Muller on the device: the same streams as keys(), but the device's
        # log/cos may round differently from numpy's in the last place
        z2 = splitmix64_torch(seed ^ 0xC3C3C3C3C3C3C3C3, n, device)
        u1 = (((z >> 11) & ((1 << 53) - 1)).to(torch.float64) + 1.0) * (2.0 ** -53)
        u2 = ((z2 >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
        g = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * torch.pi * u2)
        return g.to(torch.float32 if dtype == "float32" else torch.float64)
    raise ValueError("keys_torch supports uniform, sorted, reverse, few_unique and gaussian")


def _uniform_bits_torch(dtype, z):
    import torch
    if dtype in ("int32", "uint32"):
        hi = (z >> 32) & 0xFFFFFFFF                      # the upper 32 bits, as 0..2^32-1
        return (hi - ((hi >> 31) << 32)).to(torch.int32)  # reinterpreted as int32
    if dtype in ("int64", "uint64"):
        return z
    if dtype == "float32":
        return ((z >> 40) & 0xFFFFFF).to(torch.float32) * (2.0 ** -24)
    if dtype == "float64":
        return ((z >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
    raise ValueError(dtype)


def _sort_like_numpy(k, dtype):
    import torch
    if dtype == "uint32":
        return k[torch.argsort(k.to(torch.int64) & 0xFFFFFFFF, stable=True)]
    if dtype == "uint64":
        return k[torch.argsort(k ^ (-(1 << 63)), stable=True)]
    return torch.sort(k, stable=True)[0]

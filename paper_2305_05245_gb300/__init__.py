"""GB300-native parallel samplesort (Tokuue & Ishiyama, arXiv 2305.05245, Sec. 2).

Thin Python binding over the C ABI of ``libpsort.so`` (include/psort.h).
Every function here only marshals arguments: torch provides device memory
and streams, and each step of the sort runs in the library's CUDA kernels.

    import torch, paper_2305_05245_gb300 as ps
    x = torch.randint(-2**31, 2**31, (1 << 20,), dtype=torch.int32, device="cuda")
    ps.sort(x, "exact")            # in place, on the current stream
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _lib
from ._lib import PS_PIVOT_EXACT, PS_PIVOT_REGULAR, PsortError  # noqa: F401

__all__ = ["sort", "sort_pairs", "sort_host", "resolve_params", "workspace_bytes", "Trace",
           "PsortError", "PS_PIVOT_EXACT", "PS_PIVOT_REGULAR", "profile_enable", "profile_read",
           "profile_reset", "sort_noalloc", "sort_batch", "sort_struct", "Server", "BatchPlan", "autotune",
           "autotune_table", "autotune_set"]

_MODES = {"regular": _lib.PS_PIVOT_REGULAR, "psrs": _lib.PS_PIVOT_REGULAR, 0: 0,
          "exact": _lib.PS_PIVOT_EXACT, "pses": _lib.PS_PIVOT_EXACT, 1: 1}


def _dtype_code(dt) -> int:
    import torch
    m = {torch.int32: _lib.PS_I32, torch.int64: _lib.PS_I64, torch.float32: _lib.PS_F32,
         torch.float64: _lib.PS_F64}
    if hasattr(torch, "uint32"):
        m[torch.uint32] = _lib.PS_U32
        m[torch.uint64] = _lib.PS_U64
    if dt not in m:
        raise TypeError("unsupported key dtype %s" % dt)
    return m[dt]


def _np_dtype_code(dt) -> int:
    import numpy as np
    m = {np.dtype(np.int32): _lib.PS_I32, np.dtype(np.int64): _lib.PS_I64,
         np.dtype(np.float32): _lib.PS_F32, np.dtype(np.float64): _lib.PS_F64,
         np.dtype(np.uint32): _lib.PS_U32, np.dtype(np.uint64): _lib.PS_U64}
    return m[np.dtype(dt)]


def _mode(m) -> int:
    try:
        return _MODES[m]
    except KeyError:
        raise ValueError("pivot mode must be 'regular' or 'exact'") from None


_MERGES = {"tree": 0, "sort": 1, "select": 2, 0: 0, 1: 1, 2: 2}


def _params(n_blocks: int, n_parts: int, merge_variant="tree", items_per_thread: int = 0,
            block_threads: int = 0):
    p = _lib.PsParams()
    p.n_blocks = n_blocks
    p.n_parts = n_parts
    if merge_variant not in _MERGES:
        raise ValueError("merge_variant must be 'tree', 'sort' or 'select'")
    p.merge_variant = _MERGES[merge_variant]
    p.items_per_thread = items_per_thread
    p.block_threads = block_threads
    return p


def _stream_handle(stream) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


@dataclass
class Trace:
    """Intermediates of one sort (device tensors): pivots P_1..P_{n_P-1},
    pivot payloads (records), tie counts c_k (Eq. 2), the n_B x (n_P+1) split
    table, and the partition offsets O_0..O_{n_P}."""
    pivots: object
    pivot_payload: object
    c: object
    splits: object
    offsets: object
    n_blocks: int
    n_parts: int


def resolve_params(n: int, dtype_code: int, n_blocks: int = 0, n_parts: int = 0) -> tuple[int, int]:
    """(n_B, n_P) that a sort of n keys would use (0 = automatic)."""
    lib = _lib.load()
    out = _lib.PsParams()
    _lib.check(lib, "ps_resolve_params",
               lib.ps_resolve_params(n, dtype_code, ctypes.byref(_params(n_blocks, n_parts)),
                                     ctypes.byref(out)))
    return out.n_blocks, out.n_parts


def workspace_bytes(n: int, dtype_code: int, n_blocks: int = 0, n_parts: int = 0) -> int:
    lib = _lib.load()
    out = ctypes.c_size_t()
    _lib.check(lib, "ps_workspace_bytes",
               lib.ps_workspace_bytes(n, dtype_code, ctypes.byref(_params(n_blocks, n_parts)),
                                      ctypes.byref(out)))
    return out.value


def _make_trace(n: int, code: int, n_blocks: int, n_parts: int, key_dtype, device, records: bool):
    import torch
    nb, npart = resolve_params(n, -1 if records else code, n_blocks, n_parts)
    t = Trace(pivots=torch.zeros(max(npart - 1, 1), dtype=key_dtype, device=device),
              pivot_payload=torch.zeros(max(npart - 1, 1), dtype=torch.int32, device=device),
              c=torch.zeros(max(npart - 1, 1), dtype=torch.int64, device=device),
              splits=torch.zeros((nb, npart + 1), dtype=torch.int64, device=device),
              offsets=torch.zeros(npart + 1, dtype=torch.int64, device=device),
              n_blocks=nb, n_parts=npart)
    ct = _lib.PsTrace()
    ct.pivots = t.pivots.data_ptr()
    ct.pivot_payload = t.pivot_payload.data_ptr() if records else None
    ct.c = t.c.data_ptr()
    ct.splits = t.splits.data_ptr()
    ct.offsets = t.offsets.data_ptr()
    return t, ct


def sort(keys, pivot_mode="exact", n_blocks: int = 0, n_parts: int = 0, trace: bool = False,
         stream=None, merge_variant="tree", items_per_thread: int = 0, block_threads: int = 0):
    """Sort a contiguous 1-D CUDA tensor in place (int32, int64, float32,
    float64, uint32, uint64).  Returns a Trace when ``trace`` is true.
    ``merge_variant`` picks step 4's chunk merge: "tree" (pairwise merge
    levels, the default), "sort" (copy the pieces and sort) or "select"
    (one selection tree per chunk); all give the same result.
    ``items_per_thread`` (16, 32) and ``block_threads`` (128, 256, 512) fix
    the launch shape of the data passes (0 = automatic)."""
    lib = _lib.load()
    if not keys.is_cuda or keys.dim() != 1 or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous 1-D CUDA tensor")
    code = _dtype_code(keys.dtype)
    n = keys.numel()
    tr, ct = (None, None)
    if trace:
        tr, ct = _make_trace(n, code, n_blocks, n_parts, keys.dtype, keys.device, False)
    rc = lib.ps_sort_ex(keys.data_ptr() if n else None, n, code, _mode(pivot_mode),
                        ctypes.byref(_params(n_blocks, n_parts, merge_variant, items_per_thread,
                                             block_threads)),
                        ctypes.byref(ct) if ct is not None else None, _stream_handle(stream))
    _lib.check(lib, "ps_sort_ex", rc)
    return tr


def sort_pairs(keys, payload, pivot_mode="exact", n_blocks: int = 0, n_parts: int = 0,
               trace: bool = False, stream=None, merge_variant="tree"):
    """Sort records in place by (key, payload): ``keys`` a contiguous 1-D CUDA
    tensor of 64-bit keys (int64 storage read as unsigned), ``payload`` one of
    32-bit payloads (int32 storage read as unsigned)."""
    lib = _lib.load()
    n = keys.numel()
    if payload.numel() != n or keys.element_size() != 8 or payload.element_size() != 4:
        raise ValueError("records need 64-bit keys and 32-bit payloads of equal length")
    if not (keys.is_cuda and payload.is_cuda and keys.is_contiguous() and payload.is_contiguous()):
        raise ValueError("keys and payload must be contiguous CUDA tensors")
    tr, ct = (None, None)
    if trace:
        tr, ct = _make_trace(n, -1, n_blocks, n_parts, keys.dtype, keys.device, True)
    rc = lib.ps_sort_pairs(keys.data_ptr() if n else None, payload.data_ptr() if n else None, n,
                           _mode(pivot_mode), ctypes.byref(_params(n_blocks, n_parts, merge_variant)),
                           ctypes.byref(ct) if ct is not None else None, _stream_handle(stream))
    _lib.check(lib, "ps_sort_pairs", rc)
    return tr


def sort_struct(records, record_bytes: int | None = None, key_offset: int = 0, pivot_mode="exact",
                n_blocks: int = 0, n_parts: int = 0, stream=None) -> None:
    """Sort fixed-size records in place by the uint64 key at byte
    ``key_offset`` of each record (ps_sort_struct); equal keys keep their
    input order.  ``records`` is a contiguous CUDA tensor; ``record_bytes``
    defaults to the byte size of one row of a 2-D tensor."""
    lib = _lib.load()
    if not records.is_cuda or not records.is_contiguous():
        raise ValueError("records must be a contiguous CUDA tensor")
    nbytes = records.numel() * records.element_size()
    if record_bytes is None:
        if records.dim() != 2:
            raise ValueError("record_bytes is needed unless records is 2-D (one row per record)")
        record_bytes = records.shape[1] * records.element_size()
    if record_bytes <= 0 or nbytes % record_bytes:
        raise ValueError("the tensor is not a whole number of records")
    n = nbytes // record_bytes
    rc = lib.ps_sort_struct(records.data_ptr() if n else None, n, record_bytes, key_offset, _mode(pivot_mode),
                            ctypes.byref(_params(n_blocks, n_parts)), _stream_handle(stream))
    _lib.check(lib, "ps_sort_struct", rc)


def _code_of(dtype) -> int:
    import torch
    if isinstance(dtype, int):
        return dtype
    if isinstance(dtype, str):
        dtype = getattr(torch, dtype)
    return _dtype_code(dtype)


def autotune(dtype, pivot_mode="exact", n_min: int = 1 << 14, n_max: int = 1 << 26, batched: bool = False,
             stream=None) -> dict:
    """Run the library's autotuner (ps_autotune) for keys of ``dtype``'s width
    over the power-of-two sizes in [n_min, n_max]; returns the tuned table
    {log2 n: (n_blocks, n_parts, items_per_thread, block_threads)} that
    automatic parameters now use (a shape of 0, 0 is the automatic one)."""
    lib = _lib.load()
    code = _code_of(dtype)
    rc = lib.ps_autotune(code, _mode(pivot_mode), n_min, n_max, 1 if batched else 0, _stream_handle(stream))
    _lib.check(lib, "ps_autotune", rc)
    return autotune_table(dtype, batched)


def autotune_table(dtype, batched: bool = False) -> dict:
    """The tuned entries {log2 n: (n_blocks, n_parts, items_per_thread,
    block_threads)} for ``dtype``'s width."""
    lib = _lib.load()
    code = _code_of(dtype)
    out = {}
    for b in range(64):
        p = _lib.PsParams()
        if lib.ps_autotune_get(code, 1 if batched else 0, b, ctypes.byref(p)) == 0:
            out[b] = (p.n_blocks, p.n_parts, p.items_per_thread, p.block_threads)
    return out


def autotune_set(dtype, log2_n: int, n_blocks: int, n_parts: int, batched: bool = False,
                 items_per_thread: int = 0, block_threads: int = 0) -> None:
    """Write (or, with zeros, clear) one tuned entry, e.g. to restore a saved table."""
    lib = _lib.load()
    p = _lib.PsParams()
    p.n_blocks, p.n_parts = n_blocks, n_parts
    p.items_per_thread, p.block_threads = items_per_thread, block_threads
    _lib.check(lib, "ps_autotune_set", lib.ps_autotune_set(_code_of(dtype), 1 if batched else 0, log2_n,
                                                            ctypes.byref(p)))


def sort_host(arr, pivot_mode="exact", n_blocks: int = 0, n_parts: int = 0, stream=None) -> None:
    """Sort a host array in place through ps_sort_host and wait.  ``arr`` is a
    contiguous numpy array or a CPU torch tensor; pinned (page-locked) memory
    is read and written by the sort's first and last passes directly, other
    memory is copied to the device and back."""
    lib = _lib.load()
    import numpy as np
    if isinstance(arr, np.ndarray):
        if not arr.flags["C_CONTIGUOUS"]:
            raise ValueError("host array must be contiguous")
        code, ptr, n = _np_dtype_code(arr.dtype), arr.ctypes.data, arr.size
    else:
        if arr.is_cuda or not arr.is_contiguous():
            raise ValueError("host tensor must be a contiguous CPU tensor")
        code, ptr, n = _dtype_code(arr.dtype), arr.data_ptr(), arr.numel()
    rc = lib.ps_sort_host(ptr if n else None, n, code, _mode(pivot_mode),
                          ctypes.byref(_params(n_blocks, n_parts)), _stream_handle(stream))
    _lib.check(lib, "ps_sort_host", rc)


def profile_enable(on: bool = True) -> bool:
    """Record per-kernel CUDA events around every library launch."""
    return bool(_lib.load().ps_profile_enable(1 if on else 0))


def profile_reset() -> None:
    _lib.check(_lib.load(), "ps_profile_reset", _lib.load().ps_profile_reset())


def profile_read() -> dict:
    """{kernel label: (launches, total device ms)} since the last reset."""
    lib = _lib.load()
    cap = 64
    buf = (_lib.PsKernelStat * cap)()
    n = ctypes.c_int()
    _lib.check(lib, "ps_profile_read", lib.ps_profile_read(buf, cap, ctypes.byref(n)))
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(min(n.value, cap))}


def sort_noalloc(keys, pivot_mode="exact", stream=None) -> None:
    """Sort in place through ps_sort_noalloc, the entry point that takes its
    workspace from the library's static device array instead of allocating
    (for callers that may not allocate device memory; at most
    PS_NOALLOC_MAX_KEYS keys, and concurrent calls must be serialised)."""
    lib = _lib.load()
    if not keys.is_cuda or keys.dim() != 1 or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous 1-D CUDA tensor")
    n = keys.numel()
    rc = lib.ps_sort_noalloc(keys.data_ptr() if n else None, n, _dtype_code(keys.dtype),
                             _mode(pivot_mode), _stream_handle(stream))
    _lib.check(lib, "ps_sort_noalloc", rc)


def sort_batch(keys, seg_offsets, pivot_mode="exact", stream=None) -> None:
    """Sort every segment keys[seg_offsets[i]:seg_offsets[i+1]] in place with
    one batched call (ps_sort_batch).  ``seg_offsets`` is an int64 CUDA tensor
    of n_segs+1 non-decreasing offsets."""
    lib = _lib.load()
    if not keys.is_cuda or keys.dim() != 1 or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous 1-D CUDA tensor")
    import torch
    if seg_offsets.dtype != torch.int64 or not seg_offsets.is_cuda or not seg_offsets.is_contiguous():
        raise ValueError("seg_offsets must be a contiguous int64 CUDA tensor")
    n_segs = seg_offsets.numel() - 1
    if n_segs < 1:
        return
    rc = lib.ps_sort_batch(seg_offsets.data_ptr(), n_segs, keys.data_ptr() if keys.numel() else None,
                           _dtype_code(keys.dtype), _mode(pivot_mode), _stream_handle(stream))
    _lib.check(lib, "ps_sort_batch", rc)


class BatchPlan:
    """A batch shape planned once (ps_batch_plan_create): ``run`` sorts every
    segment of a key tensor laid out by the same offsets with no host
    synchronisation or allocation, so it can be captured in a CUDA graph.

        plan = BatchPlan(offsets_numpy_int64, torch.int32, "exact")
        plan.run(keys)                       # or inside torch.cuda.graph(...)
        plan.close()"""

    def __init__(self, seg_offsets, dtype, pivot_mode="exact"):
        import numpy as np
        self._lib = _lib.load()
        off = np.ascontiguousarray(np.asarray(seg_offsets, dtype=np.int64))
        self._code = _code_of(dtype)
        h = ctypes.c_void_p()
        _lib.check(self._lib, "ps_batch_plan_create",
                   self._lib.ps_batch_plan_create(off.ctypes.data if off.size else None, max(off.size - 1, 0),
                                                  self._code, _mode(pivot_mode), ctypes.byref(h)))
        self._h = h
        self.extent = int(off[-1]) if off.size else 0

    def run(self, keys, stream=None) -> None:
        if not keys.is_cuda or keys.dim() != 1 or not keys.is_contiguous():
            raise ValueError("keys must be a contiguous 1-D CUDA tensor")
        if keys.element_size() != (4 if self._code in (0, 2, 4) else 8):
            raise ValueError("keys do not have the plan's key width")
        if keys.numel() < self.extent:
            raise ValueError("keys are shorter than the planned segments")
        _lib.check(self._lib, "ps_batch_run", self._lib.ps_batch_run(self._h, keys.data_ptr(), _stream_handle(stream)))

    def close(self) -> None:
        if self._h:
            _lib.check(self._lib, "ps_batch_plan_destroy", self._lib.ps_batch_plan_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Sort server with continuous batching (ps_server_*).

        srv = Server(budget_bytes=32 << 30, max_inflight=4096)
        rid = srv.submit(tensor, "exact")   # tensor sorted in place later
        for rid, status in srv.poll(): ...
        srv.close()

    The tensor must be ready (synchronise its stream) before submit and must
    stay alive and untouched until its id comes back from poll()."""

    def __init__(self, budget_bytes: int, max_inflight: int = 1024):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(self._lib, "ps_server_open",
                   self._lib.ps_server_open(budget_bytes, max_inflight, ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, keys, pivot_mode="exact", code: int | None = None) -> int:
        if not keys.is_cuda or keys.dim() != 1 or not keys.is_contiguous():
            raise ValueError("keys must be a contiguous 1-D CUDA tensor")
        rid = ctypes.c_uint64()
        n = keys.numel()
        rc = self._lib.ps_server_submit(self._h, keys.data_ptr() if n else None, n,
                                        _dtype_code(keys.dtype) if code is None else code,
                                        _mode(pivot_mode), ctypes.byref(rid))
        _lib.check(self._lib, "ps_server_submit", rc)
        self._keep[rid.value] = keys
        return rid.value

    def poll(self, cap: int = 4096):
        ids = (ctypes.c_uint64 * cap)()
        st = (ctypes.c_int * cap)()
        n = ctypes.c_int()
        _lib.check(self._lib, "ps_server_poll", self._lib.ps_server_poll(self._h, ids, st, cap, ctypes.byref(n)))
        out = [(ids[i], st[i]) for i in range(n.value)]
        for rid, _ in out:
            self._keep.pop(rid, None)
        return out

    def debug_fail(self, what: str, count: int = 1) -> None:
        """Host-side failure injection (ps_server_debug_fail): "rounds" fails the
        next admitted rounds at launch, "streams" retires idle stream slots."""
        code = {"rounds": 0, "streams": 1}[what]
        _lib.check(self._lib, "ps_server_debug_fail", self._lib.ps_server_debug_fail(self._h, code, count))

    def close(self) -> None:
        if self._h:
            _lib.check(self._lib, "ps_server_close", self._lib.ps_server_close(self._h))
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""ctypes view of libpsort.so (the C ABI of include/psort.h).

Loading fails loudly when the library has not been built: there is no
Python or CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpsort.so")

PS_OK = 0
STATUS = {0: "PS_OK", -1: "PS_ERR_INVALID_ARG", -2: "PS_ERR_UNSUPPORTED", -3: "PS_ERR_NO_MEMORY",
          -4: "PS_ERR_CUDA", -5: "PS_ERR_BUSY", -6: "PS_ERR_TIMEOUT", -7: "PS_ERR_NOT_FOUND"}

PS_I32, PS_I64, PS_F32, PS_F64, PS_U32, PS_U64 = range(6)
PS_PIVOT_REGULAR, PS_PIVOT_EXACT = 0, 1

# every symbol include/psort.h declares
EXPORTS = ["ps_sort", "ps_sort_ex", "ps_sort_pairs", "ps_sort_host", "ps_resolve_params",
           "ps_workspace_bytes", "ps_status_string", "ps_last_cuda_error", "ps_profile_enable",
           "ps_profile_read", "ps_profile_reset", "ps_sort_noalloc", "ps_debug_violation", "ps_sort_batch",
           "ps_server_open", "ps_server_submit", "ps_server_poll", "ps_server_close", "ps_sort_struct",
           "ps_autotune", "ps_autotune_get", "ps_autotune_set", "ps_server_debug_fail",
           "ps_batch_plan_create", "ps_batch_run", "ps_batch_plan_destroy", "ps_debug_fail_alloc"]

PS_NOALLOC_MAX_KEYS = 1 << 20
PS_NOALLOC_SCRATCH_BYTES = 12 << 20
PS_STRUCT_MAX_BYTES = 4096


class PsParams(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int64), ("n_parts", ctypes.c_int64),
                ("merge_variant", ctypes.c_int64), ("items_per_thread", ctypes.c_int32),
                ("block_threads", ctypes.c_int32)]


class PsTrace(ctypes.Structure):
    _fields_ = [("pivots", ctypes.c_void_p), ("pivot_payload", ctypes.c_void_p),
                ("c", ctypes.c_void_p), ("splits", ctypes.c_void_p), ("offsets", ctypes.c_void_p)]


class PsKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class PsortError(RuntimeError):
    def __init__(self, fn: str, status: int, lib=None):
        text = STATUS.get(status, str(status))
        if lib is not None:
            try:
                text = "%s (%s)" % (text, lib.ps_status_string(status).decode())
                if status == -4:
                    text += ", cudaError %d" % lib.ps_last_cuda_error()
            except Exception:
                pass
        super().__init__("%s failed: %s" % (fn, text))
        self.status = status


_lib = None


def load(path: str | None = None):
    """The loaded library (raises if libpsort.so is missing)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    # PSORT_LIB selects another build of the same ABI (e.g. the bounds-checked one)
    p = path or os.environ.get("PSORT_LIB") or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("libpsort.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_2305_05245_gb300.build" % p)
    lib = ctypes.CDLL(p)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.ps_sort.argtypes = [vp, i64, i32, i32, vp]
    lib.ps_sort_ex.argtypes = [vp, i64, i32, i32, ctypes.POINTER(PsParams), ctypes.POINTER(PsTrace), vp]
    lib.ps_sort_pairs.argtypes = [vp, vp, i64, i32, ctypes.POINTER(PsParams), ctypes.POINTER(PsTrace), vp]
    lib.ps_sort_host.argtypes = [vp, i64, i32, i32, ctypes.POINTER(PsParams), vp]
    lib.ps_resolve_params.argtypes = [i64, i32, ctypes.POINTER(PsParams), ctypes.POINTER(PsParams)]
    lib.ps_workspace_bytes.argtypes = [i64, i32, ctypes.POINTER(PsParams), ctypes.POINTER(ctypes.c_size_t)]
    lib.ps_status_string.argtypes = [i32]
    lib.ps_status_string.restype = ctypes.c_char_p
    lib.ps_last_cuda_error.argtypes = []
    lib.ps_sort_noalloc.argtypes = [vp, i64, i32, i32, vp]
    lib.ps_sort_batch.argtypes = [vp, i64, vp, i32, i32, vp]
    lib.ps_sort_struct.argtypes = [vp, i64, i64, i64, i32, ctypes.POINTER(PsParams), vp]
    lib.ps_autotune.argtypes = [i32, i32, i64, i64, i32, vp]
    lib.ps_autotune_get.argtypes = [i32, i32, i32, ctypes.POINTER(PsParams)]
    lib.ps_autotune_set.argtypes = [i32, i32, i32, ctypes.POINTER(PsParams)]
    lib.ps_server_open.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
    lib.ps_server_submit.argtypes = [vp, vp, i64, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
    lib.ps_server_poll.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i32), i32,
                                   ctypes.POINTER(i32)]
    lib.ps_server_close.argtypes = [vp]
    lib.ps_server_debug_fail.argtypes = [vp, i32, i32]
    lib.ps_batch_plan_create.argtypes = [vp, i64, i32, i32, ctypes.POINTER(vp)]
    lib.ps_batch_run.argtypes = [vp, vp, vp]
    lib.ps_batch_plan_destroy.argtypes = [vp]
    lib.ps_debug_fail_alloc.argtypes = [i32]
    lib.ps_debug_violation.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    lib.ps_profile_enable.argtypes = [i32]
    lib.ps_profile_read.argtypes = [ctypes.POINTER(PsKernelStat), i32, ctypes.POINTER(i32)]
    lib.ps_profile_reset.argtypes = []
    for name in ("ps_sort", "ps_sort_ex", "ps_sort_pairs", "ps_sort_host", "ps_resolve_params",
                 "ps_workspace_bytes", "ps_last_cuda_error", "ps_profile_enable", "ps_profile_read",
                 "ps_profile_reset", "ps_sort_noalloc", "ps_debug_violation", "ps_sort_batch", "ps_server_open",
                 "ps_server_submit", "ps_server_poll", "ps_server_close", "ps_sort_struct", "ps_autotune",
                 "ps_autotune_get", "ps_autotune_set", "ps_server_debug_fail", "ps_batch_plan_create",
                 "ps_batch_run", "ps_batch_plan_destroy", "ps_debug_fail_alloc"):
        getattr(lib, name).restype = i32
    if path is None:
        _lib = lib
    return lib


def check(lib, fn: str, status: int) -> None:
    if status != PS_OK:
        raise PsortError(fn, status, lib)

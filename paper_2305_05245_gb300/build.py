"""Compile libpsort.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

The translation units are compiled in parallel with nvcc and linked into
``paper_2305_05245_gb300/libpsort.so``.  Nothing here runs on the GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpsort.so")
LIB_CHECKED = os.path.join(HERE, "libpsort_checked.so")
BUILD = os.path.join(HERE, "_build")

SOURCES = ["psort_u32.cu", "psort_u64.cu", "psort_rec.cu", "psort_api.cu", "psort_noalloc.cu",
           "psort_server.cu", "psort_struct.cu", "psort_shapes.cu"]
# Launch shapes (key bits, items per thread, threads per CTA) compiled besides
# the automatic one, each from psort_shape.cu into an object of its own; the
# 64-bit (32, 256) shape is the automatic one and is not repeated.
SHAPES = [(b, e, t) for b in (32, 64) for e in (16, 32) for t in (128, 256, 512)
          if (b, e, t) != (64, 32, 256)]


def units():
    """(source, object name, extra flags) of every translation unit."""
    out = [(src, src.replace(".cu", ".o"), []) for src in SOURCES]
    for b, e, t in SHAPES:
        out.append(("psort_shape.cu", "psort_shape_u%d_e%d_t%d.o" % (b, e, t),
                    ["-DPS_SHAPE_BITS=%d" % b, "-DPS_SHAPE_ITEMS=%d" % e, "-DPS_SHAPE_THREADS=%d" % t]))
    return out
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpsort")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "psort.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libpsort.so if it is missing or older than its sources.  With
    checked=True, build libpsort_checked.so instead: every kernel index is
    validated and violations are recorded (ps_debug_violation)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    extra = ["-DPS_CHECKED"] if checked else []

    def compile_one(unit):
        src, name, flags = unit
        obj = os.path.join(bdir, name)
        cmd = [cc, *ARCH, *FLAGS, *extra, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (name, r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    todo = units()
    with cf.ThreadPoolExecutor(max_workers=min(len(todo), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, todo))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))

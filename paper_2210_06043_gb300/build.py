"""Builds the CUDA library ``liblbib.so`` in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel; the result is linked as a
shared library with the static CUDA runtime, so it loads into any process
(PyTorch's or not) that has the driver.

``build(checked=True)`` makes the bounds-checked debug build
``liblbib_checked.so`` (``-DLBIB_CHECKED``): the kernels' population, node,
tile and marker indices are checked against their arrays, an index outside
sets a status bit that the next sync reports as LBIB_ERR_STATE, and the access
is redirected to the array's first element (nothing traps).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbib.so")
LIB_CHECKED = os.path.join(OUT_DIR, "liblbib_checked.so")
SOURCES = ("lbib_api.cu", "lbib_lbm.cu", "lbib_lag.cu", "lbib_lag_mls.cu", "lbib_noalloc.cu", "lbib_mlp.cu")
HEADERS = ("lbib_internal.cuh", "lbib_device.cuh", "lbib_lag_kernel.cuh", "lbib_trace.h")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build liblbib)")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(HERE, "..", "include", "lbib.h"))
    deps.append(os.path.join(HERE, "..", "include", "lbib_mlp.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(p) > t for p in deps)


def flags(extra=()):
    return ["-O3", ARCH, "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-O3", *extra]


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Compile (if stale) and return the path of liblbib.so (liblbib_checked.so
    with ``checked``)."""
    lib = LIB_CHECKED if checked else LIB
    if checked:
        extra = (*extra, "-DLBIB_CHECKED")
    if not force and not _stale(lib):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    tag = f"{os.getpid()}{'c' if checked else ''}"
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", f".{tag}.o"))
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj, *flags(extra)]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    try:
        with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            for obj, log in ex.map(compile_one, SOURCES):
                objs.append(obj)
                if verbose and log:
                    print(log)
    finally:  # a failed compile leaves no objects behind
        if len(objs) < len(SOURCES):
            for src in SOURCES:
                o = os.path.join(OUT_DIR, src.replace(".cu", f".{tag}.o"))
                if os.path.exists(o):
                    os.remove(o)
    tmp = lib + f".{tag}.tmp"
    r = subprocess.run([cc, "-shared", ARCH, "-o", tmp, *objs], capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))

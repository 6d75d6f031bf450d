"""Build ``libfora.so`` (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

The translation units compile in parallel and link into
``paper_1908_10583_gb300/_build/libfora.so`` (static CUDA runtime).  Set
``FORA_PTXAS_VERBOSE=1`` to print the register and shared-memory use of every
kernel.  ``build(debug=True)`` builds ``_build/debug/libfora_debug.so`` with
``-DFORA_DEBUG`` (device index checks that report FORA_ERR_BOUNDS); the package
loads it instead of the normal library when ``FORA_LIB_DEBUG=1`` is set.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libfora.so")
DEBUG_DIR = os.path.join(BUILD_DIR, "debug")
DEBUG_LIB_PATH = os.path.join(DEBUG_DIR, "libfora_debug.so")
SOURCES = ["push.cu", "walk.cu", "topk.cu", "capi.cu", "topk_noalloc.cu", "learn.cu", "server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _flags():
    f = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
         "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]
    if os.environ.get("FORA_PTXAS_VERBOSE"):
        f += ["-Xptxas", "-v"]
    return f


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, "fora_engine.cuh"), os.path.join(CSRC, "runtime.h"),
              os.path.join(INCLUDE, "fora.h"), __file__]
    return files


def up_to_date(lib: str = LIB_PATH) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every CUDA translation unit and link libfora.so (or, with debug, the
    FORA_DEBUG library); returns its path."""
    lib = DEBUG_LIB_PATH if debug else LIB_PATH
    out_dir = DEBUG_DIR if debug else BUILD_DIR
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = _flags() + (["-DFORA_DEBUG"] if debug else [])

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj, *flags]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr}")
        if verbose or os.environ.get("FORA_PTXAS_VERBOSE"):
            print(res.stderr, end="")
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lpthread", "-ldl"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))

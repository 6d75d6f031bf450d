"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Holds none of the query method's arithmetic: it generates directed R-MAT
graphs (int32 CSR, the stand-in for the social graphs of the paper's
Section 8) and uniform query sources.  The generator itself is plain C
(``rmat.c``), compiled here with gcc and loaded with ctypes.

Recipe: R-MAT quadrant probabilities (a, b, c, d) = (0.57, 0.19, 0.19, 0.05),
n = 2^scale nodes, n*avg_deg raw edges (duplicates and self-loops kept),
seeded uniform id relabelling, one extra edge to a uniform node for every
node without out-edges, rows sorted ascending.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmat.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "librmat.so")
_lock = threading.Lock()
_lib = None

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def build(force: bool = False) -> str:
    """Compile the generator into ``inputs/_build/librmat.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                           _SRC, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.rmat_generate.restype = ctypes.c_int
            lib.rmat_generate.argtypes = [
                ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)),
                ctypes.POINTER(ctypes.c_int64)]
            lib.rmat_free.restype = None
            lib.rmat_free.argtypes = [ctypes.c_void_p]
            lib.uniform_sources.restype = ctypes.c_int
            lib.uniform_sources.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                            ctypes.c_void_p]
            _lib = lib
    return _lib


def rmat_csr(scale: int, avg_deg: float, seed: int, abcd=RMAT_ABCD,
             nthreads: int | None = None):
    """Return ``(row_ptr int64[n+1], col int32[m])`` of a seeded R-MAT graph."""
    lib = _load()
    a, b, c, _ = abcd
    if nthreads is None:
        nthreads = max(1, min(64, os.cpu_count() or 1))
    rp = ctypes.POINTER(ctypes.c_int64)()
    cp = ctypes.POINTER(ctypes.c_int32)()
    m = ctypes.c_int64(0)
    rc = lib.rmat_generate(int(scale), float(avg_deg), a, b, c, int(seed), int(nthreads),
                           ctypes.byref(rp), ctypes.byref(cp), ctypes.byref(m))
    if rc != 0:
        raise RuntimeError(f"rmat_generate failed with code {rc}")
    n = 1 << scale
    try:
        row_ptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
        col = np.ctypeslib.as_array(cp, shape=(m.value,)).copy()
    finally:
        lib.rmat_free(ctypes.cast(rp, ctypes.c_void_p))
        lib.rmat_free(ctypes.cast(cp, ctypes.c_void_p))
    return row_ptr, col


def uniform_sources(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` sources drawn uniformly with replacement from ``[0, n)``."""
    lib = _load()
    out = np.empty(count, dtype=np.int32)
    rc = lib.uniform_sources(int(n), int(count), int(seed), out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"uniform_sources failed with code {rc}")
    return out


def csr_from_edges(n: int, edges):
    """CSR (rows sorted) from an explicit edge list; for hand-built test graphs."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    order = np.lexsort((e[:, 1], e[:, 0]))
    e = e[order]
    deg = np.bincount(e[:, 0], minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    return row_ptr, e[:, 1].astype(np.int32)


# Workloads (graph seed, scale, average out-degree, sources, k).
WORKLOADS = {
    "rmat14_deg8": dict(scale=14, avg_deg=8, graph_seed=1, n_sources=10, k=50),
    "rmat20_deg16": dict(scale=20, avg_deg=16, graph_seed=2, n_sources=256, k=500),
    "rmat25_deg32": dict(scale=25, avg_deg=32, graph_seed=3, n_sources=64, k=500),
}
SOURCE_SEED = 101
WALK_SEED = 0x5EED

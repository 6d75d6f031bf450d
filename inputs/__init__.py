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
import hashlib
import json
import os
import subprocess
import threading
import zlib

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


_CACHE_MAGIC = b"RMATCSR1"


def _cache_key(scale, avg_deg, seed, abcd):
    """Parameters of a generated graph and their hash (names its cache file)."""
    params = {"scale": int(scale), "avg_deg": float(avg_deg), "seed": int(seed),
              "abcd": [float(x) for x in abcd], "generator": "rmat.c"}
    text = json.dumps(params, sort_keys=True)
    return params, hashlib.sha256(text.encode()).hexdigest()[:16]


def _cache_read(path, params):
    """(row_ptr, col) from a cache file whose header matches params and whose arrays
    match the header's sizes and CRC-32; None otherwise."""
    try:
        with open(path, "rb") as f:
            if f.read(len(_CACHE_MAGIC)) != _CACHE_MAGIC:
                return None
            hlen = int.from_bytes(f.read(8), "little")
            if not 0 < hlen < 1 << 16:
                return None
            head = json.loads(f.read(hlen).decode())
            if head.get("params") != params:
                return None
            n, m = int(head["n"]), int(head["m"])
            row_ptr = np.fromfile(f, dtype=np.int64, count=n + 1)
            col = np.fromfile(f, dtype=np.int32, count=m)
    except (OSError, ValueError, KeyError):
        return None
    if len(row_ptr) != n + 1 or len(col) != m:
        return None
    crc = zlib.crc32(col.view(np.uint8), zlib.crc32(row_ptr.view(np.uint8)))
    if crc != head.get("crc32") or row_ptr[0] != 0 or row_ptr[-1] != m:
        return None
    return row_ptr, col


def _cache_write(path, params, row_ptr, col):
    """Write the cache file atomically (a temporary name, then a rename)."""
    crc = zlib.crc32(col.view(np.uint8), zlib.crc32(row_ptr.view(np.uint8)))
    head = json.dumps({"params": params, "n": len(row_ptr) - 1, "m": len(col),
                       "crc32": crc}).encode()
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(_CACHE_MAGIC)
        f.write(len(head).to_bytes(8, "little"))
        f.write(head)
        row_ptr.tofile(f)
        col.tofile(f)
    os.replace(tmp, path)


def rmat_csr(scale: int, avg_deg: float, seed: int, abcd=RMAT_ABCD,
             nthreads: int | None = None, cache_dir: str | None = None):
    """Return ``(row_ptr int64[n+1], col int32[m])`` of a seeded R-MAT graph.

    With ``cache_dir`` (default: the directory in ``FORA_GRAPH_CACHE``, if set) the graph
    is kept there as a binary CSR file behind a header holding the generator's parameters
    and a CRC-32 of the arrays, named by a hash of the parameters; a file whose header or
    checksum does not match is regenerated.  Generation is deterministic, so a cached
    graph equals a generated one."""
    if cache_dir is None:
        cache_dir = os.environ.get("FORA_GRAPH_CACHE") or None
    path = params = None
    if cache_dir:
        params, key = _cache_key(scale, avg_deg, seed, abcd)
        path = os.path.join(cache_dir, f"rmat_{int(scale)}_{key}.csr")
        got = _cache_read(path, params)
        if got is not None:
            return got
    row_ptr, col = _generate(scale, avg_deg, seed, abcd, nthreads)
    if path:
        os.makedirs(cache_dir, exist_ok=True)
        _cache_write(path, params, row_ptr, col)
    return row_ptr, col


def _generate(scale, avg_deg, seed, abcd, nthreads):
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

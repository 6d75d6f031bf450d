"""CPU oracle for the index-free FORA SSPPR query -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
under ``paper_1908_10583_gb300``) never calls it and shares no code with it.

``fora_oracle.c`` holds the query steps (parameters, Forward Push in
synchronous rounds (Alg. 1) and its balanced form (Alg. 3), the random-walk
phase of Alg. 2, estimate, exact top-k) in plain FP64 C; ``exact.py`` holds the ground truth (dense
solve and power iteration of Eq. (powerit)) in numpy/scipy.  Every function
here is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, published test vectors and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fora_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libfora_oracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", -1: "bad argument", -2: "dangling node", -3: "out of memory",
          -4: "walk count overflow", -5: "push not converged", -6: "walk cap"}


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, '?')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class PushStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("pushes", ctypes.c_int64),
                ("edge_pushes", ctypes.c_int64), ("rsum", ctypes.c_double)]


class WalkStats(ctypes.Structure):
    _fields_ = [("residual_nodes", ctypes.c_int64), ("walks", ctypes.c_int64),
                ("walk_steps", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, dbl, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
            lib.oracle_walk_scale.restype = dbl
            lib.oracle_walk_scale.argtypes = [dbl, dbl, dbl]
            lib.oracle_rmax_rule.restype = dbl
            lib.oracle_rmax_rule.argtypes = [dbl, dbl, dbl, dbl]
            lib.oracle_alpha_threshold.restype = ctypes.c_uint32
            lib.oracle_alpha_threshold.argtypes = [dbl]
            lib.oracle_philox4x32_10.restype = None
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_forward_push.restype = ctypes.c_int
            lib.oracle_forward_push.argtypes = [i64, P, P, i32, dbl, dbl, P, P, P]
            lib.oracle_forward_push_balanced.restype = ctypes.c_int
            lib.oracle_forward_push_balanced.argtypes = [i64, P, P, i32, dbl, dbl, dbl, dbl, dbl,
                                                         P, P, P, P]
            lib.oracle_walk_phase.restype = ctypes.c_int
            lib.oracle_walk_phase.argtypes = [i64, P, P, i32, dbl, dbl, u64, P, P, P, P]
            lib.oracle_walk_phase_zero_hop.restype = ctypes.c_int
            lib.oracle_walk_phase_zero_hop.argtypes = [i64, P, P, i32, dbl, dbl, u64, P, P, P, P]
            lib.oracle_estimate_zero_hop.restype = None
            lib.oracle_estimate_zero_hop.argtypes = [i64, P, P, P, dbl, P]
            lib.oracle_ssppr_zero_hop.restype = ctypes.c_int
            lib.oracle_ssppr_zero_hop.argtypes = [i64, P, P, i32, dbl, dbl, dbl,
                                                  dbl, dbl, u64, i64, P, P, P, P,
                                                  P, P, P, P, P]
            lib.oracle_topk_fora.restype = ctypes.c_int
            lib.oracle_topk_fora.argtypes = [i64, P, P, i32, dbl, dbl, dbl, dbl, u64, i64, P, P,
                                             P, P, P, P, P, P, P]
            lib.oracle_walk_index.restype = i64
            lib.oracle_walk_index.argtypes = [i64, P, P, dbl, dbl, dbl, u64, ctypes.c_uint32,
                                              ctypes.c_int, P, P, i64]
            lib.oracle_walk_phase_indexed.restype = ctypes.c_int
            lib.oracle_walk_phase_indexed.argtypes = [i64, dbl, dbl, P, P, P, ctypes.c_int, P, P,
                                                      P]
            lib.oracle_estimate.restype = None
            lib.oracle_estimate.argtypes = [i64, P, P, P]
            lib.oracle_topk.restype = ctypes.c_int
            lib.oracle_topk.argtypes = [i64, P, i64, P, P]
            lib.oracle_ssppr.restype = ctypes.c_int
            lib.oracle_ssppr.argtypes = [i64, P, P, i32, dbl, dbl, dbl, dbl, dbl, u64, i64,
                                         P, P, P, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data


def _graph(row_ptr, col):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return row_ptr, col, len(row_ptr) - 1


def walk_scale(eps, delta, pf):
    """C = omega / r_sum (Alg. 2)."""
    return _load().oracle_walk_scale(eps, delta, pf)


def rmax_rule(eps, delta, pf, m):
    """r_max by Eq. (rmax), with the Case 2 fallback of Section 3.2."""
    return _load().oracle_rmax_rule(eps, delta, pf, float(m))


def alpha_threshold(alpha):
    return _load().oracle_alpha_threshold(alpha)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def forward_push(row_ptr, col, s, alpha, rmax):
    """Forward Push (Alg. 1) in synchronous rounds -> (reserve, residue, PushStats)."""
    row_ptr, col, n = _graph(row_ptr, col)
    reserve = np.zeros(n)
    residue = np.zeros(n)
    st = PushStats()
    rc = _load().oracle_forward_push(n, _ptr(row_ptr), _ptr(col), int(s), alpha, rmax,
                                     _ptr(reserve), _ptr(residue), ctypes.addressof(st))
    if rc:
        raise OracleError(rc)
    return reserve, residue, st


def forward_push_balanced(row_ptr, col, s, alpha, walk_scale, cost_edge, cost_push, cost_walk):
    """Forward Push with push/walk balancing (Section 4.2, Alg. 3), synchronous rounds:
    walk_scale is C' (C, or (1 - alpha) C with zero-hop pruning), the costs are per edge
    push, per node push and per walk -> (reserve, residue, PushStats, final threshold)."""
    row_ptr, col, n = _graph(row_ptr, col)
    reserve = np.zeros(n)
    residue = np.zeros(n)
    st = PushStats()
    theta = ctypes.c_double(0.0)
    rc = _load().oracle_forward_push_balanced(n, _ptr(row_ptr), _ptr(col), int(s), alpha,
                                              walk_scale, cost_edge, cost_push, cost_walk,
                                              _ptr(reserve), _ptr(residue), ctypes.addressof(st),
                                              ctypes.addressof(theta))
    if rc:
        raise OracleError(rc)
    return reserve, residue, st, theta.value


def walk_phase(row_ptr, col, s, alpha, scale, seed, residue):
    """Random-walk phase of Alg. 2 on a given residue -> (count u32, acc u64, WalkStats)."""
    row_ptr, col, n = _graph(row_ptr, col)
    residue = np.ascontiguousarray(residue, dtype=np.float64)
    count = np.zeros(n, dtype=np.uint32)
    acc = np.zeros(n, dtype=np.uint64)
    st = WalkStats()
    rc = _load().oracle_walk_phase(n, _ptr(row_ptr), _ptr(col), int(s), alpha, scale,
                                   int(seed), _ptr(residue), _ptr(count), _ptr(acc),
                                   ctypes.addressof(st))
    if rc:
        raise OracleError(rc)
    return count, acc, st


INDEX_SOURCE = 0xFFFFFFFF  # the source id in the Philox counter of the index walks


def walk_index(row_ptr, col, alpha, scale, rmax, seed, s_index=INDEX_SOURCE, zero_hop=False):
    """FORA+ walk index (Section 3.3) -> (off int64 [n + 1], dest int32 [off[n]]): the
    ends of omega_max(v) = ceil(RN(RN(rmax d(v)) C)) walks from every v (zero-hop walks and
    their smaller omega_max with zero_hop)."""
    row_ptr, col, n = _graph(row_ptr, col)
    off = np.zeros(n + 1, dtype=np.int64)
    zh = 1 if zero_hop else 0
    total = _load().oracle_walk_index(n, _ptr(row_ptr), _ptr(col), alpha, scale, rmax, int(seed),
                                      int(s_index), zh, _ptr(off), _ptr(np.zeros(1, np.int32)), 0)
    if total < 0:
        raise OracleError(int(total))
    dest = np.zeros(max(int(total), 1), dtype=np.int32)
    got = _load().oracle_walk_index(n, _ptr(row_ptr), _ptr(col), alpha, scale, rmax, int(seed),
                                    int(s_index), zh, _ptr(off), _ptr(dest), int(total))
    if got < 0:
        raise OracleError(int(got))
    return off, dest[:total]


def walk_phase_indexed(n, scale, residue, off, dest, alpha=0.2, zero_hop=False):
    """Walk phase served from a walk index -> (count u32, acc u64, WalkStats)."""
    residue = np.ascontiguousarray(residue, dtype=np.float64)
    off = np.ascontiguousarray(off, dtype=np.int64)
    dest = np.ascontiguousarray(dest if len(dest) else np.zeros(1, np.int32), dtype=np.int32)
    count = np.zeros(n, dtype=np.uint32)
    acc = np.zeros(n, dtype=np.uint64)
    st = WalkStats()
    rc = _load().oracle_walk_phase_indexed(n, alpha, scale, _ptr(residue), _ptr(off), _ptr(dest),
                                           1 if zero_hop else 0, _ptr(count), _ptr(acc),
                                           ctypes.addressof(st))
    if rc:
        raise OracleError(rc)
    return count, acc, st


def walk_phase_zero_hop(row_ptr, col, s, alpha, scale, seed, residue):
    """Walk phase with zero-hop pruning (Section 4.1) -> (count u32, acc u64, WalkStats)."""
    row_ptr, col, n = _graph(row_ptr, col)
    residue = np.ascontiguousarray(residue, dtype=np.float64)
    count = np.zeros(n, dtype=np.uint32)
    acc = np.zeros(n, dtype=np.uint64)
    st = WalkStats()
    rc = _load().oracle_walk_phase_zero_hop(n, _ptr(row_ptr), _ptr(col), int(s), alpha, scale,
                                            int(seed), _ptr(residue), _ptr(count), _ptr(acc),
                                            ctypes.addressof(st))
    if rc:
        raise OracleError(rc)
    return count, acc, st


def estimate_zero_hop(reserve, residue, acc, alpha):
    reserve = np.ascontiguousarray(reserve, dtype=np.float64)
    residue = np.ascontiguousarray(residue, dtype=np.float64)
    acc = np.ascontiguousarray(acc, dtype=np.uint64)
    est = np.zeros(len(reserve))
    _load().oracle_estimate_zero_hop(len(reserve), _ptr(reserve), _ptr(residue), _ptr(acc),
                                     alpha, _ptr(est))
    return est


def estimate(reserve, acc):
    reserve = np.ascontiguousarray(reserve, dtype=np.float64)
    acc = np.ascontiguousarray(acc, dtype=np.uint64)
    est = np.zeros(len(reserve))
    _load().oracle_estimate(len(reserve), _ptr(reserve), _ptr(acc), _ptr(est))
    return est


def topk(est, k):
    est = np.ascontiguousarray(est, dtype=np.float64)
    ids = np.zeros(k, dtype=np.int32)
    vals = np.zeros(k)
    rc = _load().oracle_topk(len(est), _ptr(est), int(k), _ptr(ids), _ptr(vals))
    if rc:
        raise OracleError(rc)
    return ids, vals


@dataclass
class QueryResult:
    ids: np.ndarray
    vals: np.ndarray
    reserve: np.ndarray
    residue: np.ndarray
    count: np.ndarray
    acc: np.ndarray
    est: np.ndarray
    push: PushStats
    walk: WalkStats
    rmax: float


def ssppr(row_ptr, col, s, *, alpha=0.2, eps=0.5, delta=None, pf=None, rmax=0.0,
          seed=0x5EED, k=50, zero_hop=False):
    """One whole query (Alg. 2 + top-k; with zero_hop, the walk phase of Section 4.1);
    delta and p_f default to 1/n."""
    row_ptr, col, n = _graph(row_ptr, col)
    delta = 1.0 / n if delta is None else delta
    pf = 1.0 / n if pf is None else pf
    rmax_used = rmax if rmax > 0 else rmax_rule(eps, delta, pf, row_ptr[-1])
    arrays = dict(reserve=np.zeros(n), residue=np.zeros(n),
                  count=np.zeros(n, dtype=np.uint32), acc=np.zeros(n, dtype=np.uint64),
                  est=np.zeros(n))
    ids = np.zeros(k, dtype=np.int32)
    vals = np.zeros(k)
    pst, wst = PushStats(), WalkStats()
    fn = _load().oracle_ssppr_zero_hop if zero_hop else _load().oracle_ssppr
    rc = fn(n, _ptr(row_ptr), _ptr(col), int(s), alpha, eps, delta, pf,
                              rmax_used, int(seed), int(k), _ptr(arrays["reserve"]),
                              _ptr(arrays["residue"]), _ptr(arrays["count"]),
                              _ptr(arrays["acc"]), _ptr(arrays["est"]), _ptr(ids), _ptr(vals),
                              ctypes.addressof(pst), ctypes.addressof(wst))
    if rc:
        raise OracleError(rc)
    return QueryResult(ids=ids, vals=vals, push=pst, walk=wst, rmax=rmax_used, **arrays)


@dataclass
class TopkResult:
    ids: np.ndarray
    vals: np.ndarray
    est: np.ndarray
    iterations: int
    delta: float


def topk_fora(row_ptr, col, s, k, *, alpha=0.2, eps=0.5, pf=None, rmax=0.0, seed=0x5EED):
    """Top-k FORA (Alg. 5): delta halving from 1/k to 1/n with eps/2 and p_f/(n log2(n/k))."""
    row_ptr, col, n = _graph(row_ptr, col)
    pf = 1.0 / n if pf is None else pf
    work = [np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.uint32), np.zeros(n, dtype=np.uint64),
            np.zeros(n)]
    ids = np.zeros(k, dtype=np.int32)
    vals = np.zeros(k)
    it = ctypes.c_int32(0)
    dl = ctypes.c_double(0.0)
    rc = _load().oracle_topk_fora(n, _ptr(row_ptr), _ptr(col), int(s), alpha, eps, pf, rmax,
                                  int(seed), int(k), *[_ptr(a) for a in work], _ptr(ids),
                                  _ptr(vals), ctypes.addressof(it), ctypes.addressof(dl))
    if rc:
        raise OracleError(rc)
    return TopkResult(ids=ids, vals=vals, est=work[4], iterations=it.value, delta=dl.value)

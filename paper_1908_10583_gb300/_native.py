"""ctypes binding of ``libfora.so`` (include/fora.h): argument marshalling only.

Every step of a query runs in the CUDA library; this module converts numpy
arrays / torch tensors to pointers and checks return codes.  If the library
has not been built, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

FORA_OK = 0
FORA_ERR_BAD_ARG = -1
FORA_ERR_DANGLING = -2
FORA_ERR_OOM = -3
FORA_ERR_WALK_OVERFLOW = -4
FORA_ERR_PUSH_NOT_CONVERGED = -5
FORA_ERR_WALK_CAP = -6
FORA_ERR_CUDA = -7
FORA_ERR_TIMEOUT = -8
FORA_ERR_BOUNDS = -9
FORA_MAX_K = 4096
FORA_OUT_DEVICE = 0x1
FORA_ASYNC = 0x2
FORA_ZERO_HOP = 0x4
FORA_USE_INDEX = 0x8
FORA_DBG_GIVEN_PUSH = 0x1
FORA_NUM_FEATURES = 16
FORA_MODEL_PARAMS = 5313

_lock = threading.Lock()
_lib = None


class FORAError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fora error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    """fora_params: alpha, eps, delta/pf (<= 0: 1/n), rmax (<= 0: rule), k, flags, seed."""
    _fields_ = [("alpha", ctypes.c_double), ("eps", ctypes.c_double),
                ("delta", ctypes.c_double), ("pf", ctypes.c_double),
                ("rmax", ctypes.c_double), ("k", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("seed", ctypes.c_uint64)]

    @classmethod
    def make(cls, alpha=0.2, eps=0.5, delta=0.0, pf=0.0, rmax=0.0, k=50, flags=0, seed=0x5EED):
        return cls(alpha, eps, delta, pf, rmax, k, flags, seed)


class Stats(ctypes.Structure):
    _fields_ = [("rmax", ctypes.c_double), ("rsum", ctypes.c_double),
                ("pushes", ctypes.c_uint64), ("edge_pushes", ctypes.c_uint64),
                ("residual_nodes", ctypes.c_uint64), ("walks", ctypes.c_uint64),
                ("walk_steps", ctypes.c_uint64), ("push_rounds", ctypes.c_uint32),
                ("source", ctypes.c_int32), ("ms_push", ctypes.c_float),
                ("ms_residual", ctypes.c_float), ("ms_walk", ctypes.c_float),
                ("ms_topk", ctypes.c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_uint64), ("lanes_per_graph", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("batch_window_ms", ctypes.c_double),
                ("admit_during_push", ctypes.c_int32), ("pad", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("submit_ms", ctypes.c_double), ("start_ms", ctypes.c_double),
                ("end_ms", ctypes.c_double), ("batch_size", ctypes.c_uint32),
                ("lane", ctypes.c_int32), ("joined", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("stats", Stats)]


class Balance(ctypes.Structure):
    """fora_balance: costs of one edge push, one node push and one walk (Alg. 3)."""
    _fields_ = [("edge_push", ctypes.c_double), ("push", ctypes.c_double),
                ("walk", ctypes.c_double)]


class DebugIO(ctypes.Structure):
    _fields_ = [("reserve", ctypes.c_void_p), ("residue", ctypes.c_void_p),
                ("count", ctypes.c_void_p), ("acc", ctypes.c_void_p),
                ("estimate", ctypes.c_void_p), ("balance", ctypes.c_void_p)]


def lib_path() -> str:
    """The library this process loads: the FORA_DEBUG build when FORA_LIB_DEBUG=1."""
    return _build.DEBUG_LIB_PATH if os.environ.get("FORA_LIB_DEBUG") == "1" else _build.LIB_PATH


def load():
    """Load libfora.so (build it first with ``paper_1908_10583_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: the CUDA library must be built "
                               "(paper_1908_10583_gb300.build.build()); there is no CPU fallback")
        L = ctypes.CDLL(path)
        P, I, i64, i32, u32 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int32,
                               ctypes.c_uint32)
        L.fora_graph_create.restype = I
        L.fora_graph_create.argtypes = [i64, P, P, u32, ctypes.POINTER(P)]
        L.fora_graph_destroy.restype = None
        L.fora_graph_destroy.argtypes = [P]
        L.fora_graph_info.restype = I
        L.fora_graph_info.argtypes = [P, P, P, P]
        L.fora_resolve_params.restype = I
        L.fora_resolve_params.argtypes = [P, ctypes.POINTER(Params), P, P, P]
        L.fora_ssppr.restype = I
        L.fora_ssppr.argtypes = [P, ctypes.POINTER(Params), i32, P, P, P, P]
        L.fora_ssppr_batch.restype = I
        L.fora_ssppr_batch.argtypes = [P, ctypes.POINTER(Params), P, i32, P, P, P, P]
        L.fora_ssppr_batch_debug.restype = I
        L.fora_ssppr_batch_debug.argtypes = [P, ctypes.POINTER(Params), P, i32, P, P, P,
                                             ctypes.POINTER(DebugIO), u32, P]
        L.fora_ssppr_batch_balanced.restype = I
        L.fora_ssppr_batch_balanced.argtypes = [P, ctypes.POINTER(Params), ctypes.POINTER(Balance),
                                                P, i32, P, P, P, P]
        L.fora_ssppr_batch_rmax.restype = I
        L.fora_ssppr_batch_rmax.argtypes = [P, ctypes.POINTER(Params), P, P, i32, P, P, P, P]
        L.fora_topk_ssppr_batch.restype = I
        L.fora_topk_ssppr_batch.argtypes = [P, ctypes.POINTER(Params), P, i32, P, P, P, P, P]
        L.fora_topk.restype = I
        L.fora_topk.argtypes = [P, i64, i32, u32, P, P, P]
        L.fora_philox_debug.restype = I
        L.fora_philox_debug.argtypes = [P, P, i32]
        L.fora_threshold_debug.restype = I
        L.fora_threshold_debug.argtypes = [P, P, P, P, i32]
        L.fora_topk_noalloc.restype = I
        L.fora_topk_noalloc.argtypes = [P, i64, i32, u32, P, P, P]
        L.fora_model_create.restype = I
        L.fora_model_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(P)]
        L.fora_model_destroy.restype = None
        L.fora_model_destroy.argtypes = [P]
        L.fora_model_get.restype = I
        L.fora_model_get.argtypes = [P, P, P]
        L.fora_model_set.restype = I
        L.fora_model_set.argtypes = [P, P, P]
        L.fora_model_predict.restype = I
        L.fora_model_predict.argtypes = [P, P, i32, P]
        L.fora_model_gradient.restype = I
        L.fora_model_gradient.argtypes = [P, P, P, i32, P, P]
        L.fora_model_train.restype = I
        L.fora_model_train.argtypes = [P, P, P, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, P]
        L.fora_source_features.restype = I
        L.fora_source_features.argtypes = [P, ctypes.POINTER(Params), P, i32, P]
        L.fora_ssppr_batch_learned.restype = I
        L.fora_ssppr_batch_learned.argtypes = [P, ctypes.POINTER(Params), P, P, i32, P, P, P, P]
        L.fora_server_create.restype = I
        L.fora_server_create.argtypes = [P, i32, ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]
        L.fora_server_destroy.restype = None
        L.fora_server_destroy.argtypes = [P]
        L.fora_server_lane_capacity.restype = I
        L.fora_server_lane_capacity.argtypes = [P, i32, P, P]
        L.fora_server_submit.restype = I
        L.fora_server_submit.argtypes = [P, i32, i32, ctypes.POINTER(Params), P]
        L.fora_server_wait.restype = I
        L.fora_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_double, P, P, P]
        L.fora_server_stats.restype = I
        L.fora_server_stats.argtypes = [P, P, P, P, P]
        L.fora_graph_autotune.restype = I
        L.fora_graph_autotune.argtypes = [P, ctypes.POINTER(Params), P, i32, P, P, P]
        L.fora_graph_tune.restype = I
        L.fora_graph_tune.argtypes = [P, ctypes.c_char_p, i64]
        L.fora_graph_tuning.restype = I
        L.fora_graph_tuning.argtypes = [P, ctypes.c_char_p, P]
        L.fora_index_build.restype = I
        L.fora_index_build.argtypes = [P, ctypes.POINTER(Params), P]
        L.fora_index_info.restype = I
        L.fora_index_info.argtypes = [P, P, P, P]
        L.fora_index_export.restype = I
        L.fora_index_export.argtypes = [P, P, P]
        L.fora_index_destroy.restype = I
        L.fora_index_destroy.argtypes = [P]
        L.fora_workspace_bytes.restype = I
        L.fora_workspace_bytes.argtypes = [i64, P, i32, P]
        L.fora_hot_nodes.restype = I
        L.fora_hot_nodes.argtypes = [i64, P, P, P, i32, P]
        L.fora_debug_checks.restype = I
        L.fora_debug_checks.argtypes = []
        L.fora_debug_fail_alloc.restype = I
        L.fora_debug_fail_alloc.argtypes = [i64]
        L.fora_last_error.restype = ctypes.c_char_p
        L.fora_last_error.argtypes = []
        _lib = L
        return L


def header_functions():
    """Names of the functions include/fora.h declares (for the export check)."""
    text = open(os.path.join(_build.INCLUDE, "fora.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fora_[a-z0-9_]+)\s*\(", text)))


def _check(rc: int):
    if rc != FORA_OK:
        raise FORAError(rc, load().fora_last_error().decode(errors="replace"))


def _stream_ptr(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x):
    """Raw pointer of a numpy array or a torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Graph:
    """A CSR graph resident on the current CUDA device (fora_graph_create)."""

    def __init__(self, row_ptr, col):
        L = load()
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        self.n = len(row_ptr) - 1
        self.m = int(row_ptr[-1])
        h = ctypes.c_void_p()
        _check(L.fora_graph_create(self.n, row_ptr.ctypes.data, col.ctypes.data, 0,
                                   ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().fora_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, key: str, value: int):
        """Set a launch-shape parameter (fora_graph_tune); results do not depend on it."""
        _check(load().fora_graph_tune(self._h, key.encode(), int(value)))

    def build_index(self, params: Params, stream=None):
        """FORA+ walk index (fora_index_build) for these parameters."""
        _check(load().fora_index_build(self._h, ctypes.byref(params), _stream_ptr(stream)))

    def index_info(self):
        """(r_max, C, stored walks) of the walk index, zeros without one."""
        r, c, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(load().fora_index_info(self._h, ctypes.byref(r), ctypes.byref(c), ctypes.byref(e)))
        return r.value, c.value, e.value

    def index_export(self):
        """The walk index on the host: (off int64 [n + 1], dest uint32 [entries])."""
        _, _, entries = self.index_info()
        off = np.zeros(self.n + 1, dtype=np.int64)
        dest = np.zeros(max(entries, 1), dtype=np.uint32)
        _check(load().fora_index_export(self._h, off.ctypes.data, dest.ctypes.data))
        return off, dest[:entries]

    def drop_index(self):
        _check(load().fora_index_destroy(self._h))

    def tuning(self, key: str) -> int:
        """The current value of a launch-shape parameter (fora_graph_tuning)."""
        v = ctypes.c_int64()
        _check(load().fora_graph_tuning(self._h, key.encode(), ctypes.byref(v)))
        return v.value

    def autotune(self, sources, params: Params, stream=None):
        """fora_graph_autotune on a representative batch -> {spread_width, walk_blocks,
        pipeline, spread_hot}."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        sw, wb = ctypes.c_int32(), ctypes.c_int32()
        _check(load().fora_graph_autotune(self._h, ctypes.byref(params), src.ctypes.data,
                                          len(src), ctypes.byref(sw), ctypes.byref(wb),
                                          _stream_ptr(stream)))
        return {"spread_width": sw.value, "walk_blocks": wb.value,
                "pipeline": self.tuning("pipeline"), "spread_hot": self.tuning("spread_hot")}

    def info(self):
        n, m, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().fora_graph_info(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(d)))
        return n.value, m.value, d.value

    def resolve(self, params: Params):
        r, c, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint32()
        _check(load().fora_resolve_params(self._h, ctypes.byref(params), ctypes.byref(r),
                                          ctypes.byref(c), ctypes.byref(t)))
        return r.value, c.value, t.value

    def ssppr(self, source: int, params: Params, stream=None):
        """One query; host outputs. Returns (ids, vals, Stats)."""
        k = params.k
        ids = np.zeros(k, dtype=np.int32)
        vals = np.zeros(k, dtype=np.float64)
        st = Stats()
        p = Params.from_buffer_copy(params)
        p.flags &= ~FORA_OUT_DEVICE
        _check(load().fora_ssppr(self._h, ctypes.byref(p), int(source), ids.ctypes.data,
                                 vals.ctypes.data, ctypes.addressof(st), _stream_ptr(stream)))
        return ids, vals, st

    def ssppr_batch(self, sources, params: Params, out_ids=None, out_vals=None, stats=True,
                    stream=None):
        """Batched query.  With out_ids/out_vals given (torch CUDA tensors [nsrc, k]) the
        results stay on the device (FORA_OUT_DEVICE); otherwise numpy arrays are returned."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        nsrc, k = len(src), params.k
        p = Params.from_buffer_copy(params)
        if out_ids is not None:
            p.flags |= FORA_OUT_DEVICE
        else:
            p.flags &= ~FORA_OUT_DEVICE
            out_ids = np.zeros((nsrc, k), dtype=np.int32)
            out_vals = np.zeros((nsrc, k), dtype=np.float64)
        st = (Stats * nsrc)() if stats else None
        _check(load().fora_ssppr_batch(self._h, ctypes.byref(p), src.ctypes.data, nsrc,
                                       _ptr(out_ids), _ptr(out_vals),
                                       ctypes.addressof(st) if st is not None else None,
                                       _stream_ptr(stream)))
        return out_ids, out_vals, (list(st) if st is not None else None)

    def ssppr_batch_rmax(self, sources, rmax, params: Params, out_ids=None, out_vals=None,
                         stream=None):
        """Batched query with one r_max per source (host array)."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        rm = np.ascontiguousarray(rmax, dtype=np.float64)
        assert len(rm) == len(src)
        nsrc, k = len(src), params.k
        p = Params.from_buffer_copy(params)
        if out_ids is not None:
            p.flags |= FORA_OUT_DEVICE
        else:
            p.flags &= ~FORA_OUT_DEVICE
            out_ids = np.zeros((nsrc, k), dtype=np.int32)
            out_vals = np.zeros((nsrc, k), dtype=np.float64)
        st = (Stats * nsrc)()
        _check(load().fora_ssppr_batch_rmax(self._h, ctypes.byref(p), src.ctypes.data,
                                            rm.ctypes.data, nsrc, _ptr(out_ids), _ptr(out_vals),
                                            ctypes.addressof(st), _stream_ptr(stream)))
        return out_ids, out_vals, list(st)

    def ssppr_batch_balanced(self, sources, params: Params, costs, out_ids=None, out_vals=None,
                             stream=None):
        """Batched query with the balanced push of Alg. 3; costs = (edge_push, push, walk)."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        nsrc, k = len(src), params.k
        p = Params.from_buffer_copy(params)
        if out_ids is not None:
            p.flags |= FORA_OUT_DEVICE
        else:
            p.flags &= ~FORA_OUT_DEVICE
            out_ids = np.zeros((nsrc, k), dtype=np.int32)
            out_vals = np.zeros((nsrc, k), dtype=np.float64)
        st = (Stats * nsrc)()
        bal = Balance(*[float(c) for c in costs])
        _check(load().fora_ssppr_batch_balanced(self._h, ctypes.byref(p), ctypes.byref(bal),
                                                src.ctypes.data, nsrc, _ptr(out_ids),
                                                _ptr(out_vals), ctypes.addressof(st),
                                                _stream_ptr(stream)))
        return out_ids, out_vals, list(st)

    def features(self, sources, params: Params):
        """Per-source features of the learned r_max (fora_source_features) -> [nsrc, 16]."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        out = np.zeros((len(src), FORA_NUM_FEATURES), dtype=np.float32)
        _check(load().fora_source_features(self._h, ctypes.byref(params), src.ctypes.data,
                                           len(src), out.ctypes.data))
        return out

    def ssppr_batch_learned(self, sources, params: Params, model: "Model", out_ids=None,
                            out_vals=None, stream=None):
        """Batched query with r_max chosen per source by the model."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        nsrc, k = len(src), params.k
        p = Params.from_buffer_copy(params)
        if out_ids is not None:
            p.flags |= FORA_OUT_DEVICE
        else:
            p.flags &= ~FORA_OUT_DEVICE
            out_ids = np.zeros((nsrc, k), dtype=np.int32)
            out_vals = np.zeros((nsrc, k), dtype=np.float64)
        st = (Stats * nsrc)()
        _check(load().fora_ssppr_batch_learned(self._h, ctypes.byref(p), model._h,
                                               src.ctypes.data, nsrc, _ptr(out_ids),
                                               _ptr(out_vals), ctypes.addressof(st),
                                               _stream_ptr(stream)))
        return out_ids, out_vals, list(st)

    def topk_fora(self, sources, params: Params, stream=None):
        """Top-k FORA (Alg. 5) per source -> (ids [nsrc, k], vals, stats, iterations)."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        nsrc, k = len(src), params.k
        ids = np.zeros((nsrc, k), dtype=np.int32)
        vals = np.zeros((nsrc, k), dtype=np.float64)
        iters = np.zeros(nsrc, dtype=np.uint32)
        st = (Stats * nsrc)()
        p = Params.from_buffer_copy(params)
        p.flags &= ~FORA_OUT_DEVICE
        _check(load().fora_topk_ssppr_batch(self._h, ctypes.byref(p), src.ctypes.data, nsrc,
                                            ids.ctypes.data, vals.ctypes.data,
                                            ctypes.addressof(st), iters.ctypes.data,
                                            _stream_ptr(stream)))
        return ids, vals, list(st), iters

    def ssppr_batch_host(self, sources, params: Params, out_ids: np.ndarray,
                         out_vals: np.ndarray, stream=None):
        """Batched query into caller-provided host arrays ([nsrc, k] int32 / float64,
        e.g. pinned); no stats."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        p = Params.from_buffer_copy(params)
        p.flags &= ~FORA_OUT_DEVICE
        assert out_ids.dtype == np.int32 and out_vals.dtype == np.float64
        assert out_ids.size >= len(src) * p.k and out_vals.size >= len(src) * p.k
        _check(load().fora_ssppr_batch(self._h, ctypes.byref(p), src.ctypes.data, len(src),
                                       out_ids.ctypes.data, out_vals.ctypes.data, None,
                                       _stream_ptr(stream)))
        return out_ids, out_vals

    def ssppr_batch_debug(self, sources, params: Params, dbg: dict, given_push=False,
                          stream=None, balance=None):
        """Batched query exposing intermediate arrays.  dbg maps any of reserve, residue,
        count, acc, estimate to torch CUDA tensors of shape [nsrc, n]; balance = (edge_push,
        push, walk) selects the balanced push of Alg. 3."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        nsrc, k = len(src), params.k
        p = Params.from_buffer_copy(params)
        p.flags &= ~FORA_OUT_DEVICE
        ids = np.zeros((nsrc, k), dtype=np.int32)
        vals = np.zeros((nsrc, k), dtype=np.float64)
        st = (Stats * nsrc)()
        bal = Balance(*[float(c) for c in balance]) if balance is not None else None
        io = DebugIO(*[_ptr(dbg.get(f)) for f, _ in DebugIO._fields_[:5]],
                     ctypes.addressof(bal) if bal is not None else None)
        _check(load().fora_ssppr_batch_debug(self._h, ctypes.byref(p), src.ctypes.data, nsrc,
                                             ids.ctypes.data, vals.ctypes.data, ctypes.addressof(st),
                                             ctypes.byref(io),
                                             FORA_DBG_GIVEN_PUSH if given_push else 0,
                                             _stream_ptr(stream)))
        return ids, vals, list(st)


def topk(est, k: int, out_ids=None, out_vals=None, stream=None):
    """Top-k of each row of a [nrows, n] float64 CUDA tensor (fora_topk)."""
    import torch
    est = est.contiguous()
    if est.dim() == 1:
        est = est.unsqueeze(0)
    nrows, n = est.shape
    if out_ids is None:
        out_ids = torch.empty((nrows, k), dtype=torch.int32, device=est.device)
        out_vals = torch.empty((nrows, k), dtype=torch.float64, device=est.device)
    _check(load().fora_topk(est.data_ptr(), n, nrows, k, out_ids.data_ptr(), out_vals.data_ptr(),
                            _stream_ptr(stream)))
    return out_ids, out_vals


def workspace_bytes(row_ptr, nsrc: int) -> int:
    """Device bytes of a batched query of nsrc sources on this CSR (fora_workspace_bytes)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    out = ctypes.c_uint64()
    _check(load().fora_workspace_bytes(len(rp) - 1, rp.ctypes.data, int(nsrc), ctypes.byref(out)))
    return out.value


def hot_nodes(row_ptr, col) -> np.ndarray:
    """The hot nodes the push marks in this CSR graph (fora_hot_nodes, host arithmetic)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    count = ctypes.c_int32()
    _check(load().fora_hot_nodes(len(rp) - 1, rp.ctypes.data, c.ctypes.data, None, 0,
                                 ctypes.byref(count)))
    out = np.zeros(max(count.value, 1), dtype=np.int32)
    _check(load().fora_hot_nodes(len(rp) - 1, rp.ctypes.data, c.ctypes.data, out.ctypes.data,
                                 len(out), ctypes.byref(count)))
    return out[:count.value]


def debug_fail_alloc(nth: int):
    """Make the library's nth device allocation from now on fail (0: off)."""
    _check(load().fora_debug_fail_alloc(int(nth)))


def philox(ctr_key: np.ndarray) -> np.ndarray:
    """Device Philox4x32-10 on rows (ctr0..ctr3, key0, key1) -> [count, 4] words."""
    ck = np.ascontiguousarray(ctr_key, dtype=np.uint32).reshape(-1, 6)
    out = np.zeros((len(ck), 4), dtype=np.uint32)
    _check(load().fora_philox_debug(ck.ctypes.data, out.ctypes.data, len(ck)))
    return out


def threshold(r, rmax, d) -> np.ndarray:
    """The device's frontier test r > RN(rmax * d) on host arrays -> bool array."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    rm = np.ascontiguousarray(np.broadcast_to(rmax, r.shape), dtype=np.float64)
    dd = np.ascontiguousarray(np.broadcast_to(d, r.shape), dtype=np.uint32)
    out = np.zeros(r.shape, dtype=np.uint8)
    _check(load().fora_threshold_debug(r.ctypes.data, rm.ctypes.data, dd.ctypes.data,
                                       out.ctypes.data, r.size))
    return out.astype(bool)


class Model:
    """The learned r_max network (fora_model_*), resident on the current device."""

    def __init__(self, seed: int = 0):
        h = ctypes.c_void_p()
        _check(load().fora_model_create(int(seed), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().fora_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        p = np.zeros(FORA_MODEL_PARAMS, dtype=np.float32)
        nm = np.zeros(2 * FORA_NUM_FEATURES, dtype=np.float32)
        _check(load().fora_model_get(self._h, p.ctypes.data, nm.ctypes.data))
        return p, nm

    def set(self, params=None, norm=None):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        nm = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        _check(load().fora_model_set(self._h, _ptr(p), _ptr(nm)))

    def predict(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros(len(x), dtype=np.float32)
        _check(load().fora_model_predict(self._h, x.ctypes.data, len(x), y.ctypes.data))
        return y

    def gradient(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(FORA_MODEL_PARAMS, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        _check(load().fora_model_gradient(self._h, x.ctypes.data, t.ctypes.data, len(x),
                                          g.ctypes.data, ctypes.byref(loss)))
        return g, loss.value

    def train(self, x, t, epochs=50, batch=256, lr=1e-3, seed=0):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        hist = np.zeros(epochs, dtype=np.float32)
        _check(load().fora_model_train(self._h, x.ctypes.data, t.ctypes.data, len(x), int(epochs),
                                       int(batch), float(lr), int(seed), hist.ctypes.data))
        return hist

    def save(self, path):
        p, nm = self.get()
        np.savez(path, params=p, norm=nm)

    @classmethod
    def load_file(cls, path):
        d = np.load(path)
        m = cls(0)
        m.set(d["params"], d["norm"])
        return m


class Server:
    """Continuous-batching request loop over resident graphs (fora_server_*)."""

    def __init__(self, graphs, lanes_per_graph=2, max_batch=256, memory_budget_bytes=0,
                 batch_window_ms=0.5, admit_during_push=True):
        self._graphs = list(graphs)  # keep the graphs alive
        arr = (ctypes.c_void_p * len(self._graphs))(*[g._h.value for g in self._graphs])
        cfg = ServerConfig(int(memory_budget_bytes), int(lanes_per_graph), int(max_batch),
                           float(batch_window_ms), 1 if admit_during_push else 0, 0)
        h = ctypes.c_void_p()
        _check(load().fora_server_create(ctypes.cast(arr, ctypes.c_void_p), len(self._graphs),
                                         ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.lanes_per_graph = lanes_per_graph

    def close(self):
        if getattr(self, "_h", None):
            load().fora_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lane_capacity(self, lane):
        g, sl = ctypes.c_int32(), ctypes.c_int32()
        _check(load().fora_server_lane_capacity(self._h, lane, ctypes.byref(g), ctypes.byref(sl)))
        return g.value, sl.value

    def submit(self, graph: int, source: int, params: Params) -> int:
        t = ctypes.c_uint64()
        _check(load().fora_server_submit(self._h, int(graph), int(source), ctypes.byref(params),
                                         ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, k: int, timeout_ms: float = 600000.0):
        ids = np.zeros(k, dtype=np.int32)
        vals = np.zeros(k, dtype=np.float64)
        info = RequestInfo()
        _check(load().fora_server_wait(self._h, int(ticket), float(timeout_ms), ids.ctypes.data,
                                       vals.ctypes.data, ctypes.addressof(info)))
        return ids, vals, info

    def stats(self):
        c, b, m, j = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int32(), ctypes.c_uint64()
        _check(load().fora_server_stats(self._h, ctypes.byref(c), ctypes.byref(b), ctypes.byref(m),
                                        ctypes.byref(j)))
        return {"completed": c.value, "batches": b.value, "max_concurrent_lanes": m.value,
                "joined": j.value}

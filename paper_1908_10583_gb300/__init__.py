"""GB300-native index-free FORA single-source Personalized PageRank.

The query (Forward Push in synchronous rounds, the Monte-Carlo walk phase of
Alg. 2, estimate and top-k select) runs in hand-written CUDA kernels for
sm_103a behind the C ABI of ``include/fora.h``; this package is the thin
ctypes binding (``_native``) and the in-tree build (``build``).
"""
from ._native import (Balance, DebugIO, FORAError, Graph, Model, Params, Server, Stats, FORA_DBG_GIVEN_PUSH,
                      FORA_ERR_BAD_ARG, FORA_ERR_CUDA, FORA_ERR_DANGLING, FORA_ERR_OOM,
                      FORA_ERR_PUSH_NOT_CONVERGED, FORA_ERR_TIMEOUT, FORA_ERR_WALK_CAP,
                      FORA_ERR_WALK_OVERFLOW, FORA_MAX_K, FORA_OK, FORA_OUT_DEVICE, FORA_USE_INDEX,
                      FORA_ZERO_HOP, debug_fail_alloc, header_functions, hot_nodes, lib_path,
                      load, philox, threshold, topk, workspace_bytes)

__all__ = ["Balance", "DebugIO", "FORAError", "Graph", "Model", "Params", "Server", "Stats", "FORA_DBG_GIVEN_PUSH",
           "FORA_ERR_BAD_ARG", "FORA_ERR_CUDA", "FORA_ERR_DANGLING", "FORA_ERR_OOM",
           "FORA_ERR_PUSH_NOT_CONVERGED", "FORA_ERR_TIMEOUT", "FORA_ERR_WALK_CAP",
           "FORA_ERR_WALK_OVERFLOW", "FORA_MAX_K", "FORA_OK", "FORA_OUT_DEVICE", "FORA_USE_INDEX",
           "FORA_ZERO_HOP", "debug_fail_alloc", "header_functions", "hot_nodes", "lib_path", "load",
           "philox", "threshold", "topk", "workspace_bytes"]

"""Host-side checks of the C-ABI library that need no GPU."""
import os

import pytest

import paper_1908_10583_gb300 as fora
from paper_1908_10583_gb300 import build as fbuild


@pytest.fixture(scope="module")
def lib():
    fbuild.build()
    return fora.load()


def test_library_exports_every_header_function(lib):
    names = fora.header_functions()
    assert {"fora_graph_create", "fora_ssppr", "fora_ssppr_batch", "fora_last_error"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(fbuild.ARCH)
    assert os.path.exists(fbuild.LIB_PATH)


def test_bad_arguments_are_rejected_before_any_device_call(lib):
    import numpy as np
    import ctypes
    h = ctypes.c_void_p()
    # dangling node 2
    rc = lib.fora_graph_create(3, np.array([0, 1, 2, 2], dtype=np.int64).ctypes.data,
                               np.array([1, 0], dtype=np.int32).ctypes.data, 0, ctypes.byref(h))
    assert rc == fora.FORA_ERR_DANGLING
    assert b"no out-edge" in lib.fora_last_error()
    # column out of range
    rc = lib.fora_graph_create(2, np.array([0, 1, 2], dtype=np.int64).ctypes.data,
                               np.array([1, 5], dtype=np.int32).ctypes.data, 0, ctypes.byref(h))
    assert rc == fora.FORA_ERR_BAD_ARG
    # non-monotone row pointer
    rc = lib.fora_graph_create(2, np.array([0, 2, 1], dtype=np.int64).ctypes.data,
                               np.array([1, 0], dtype=np.int32).ctypes.data, 0, ctypes.byref(h))
    assert rc == fora.FORA_ERR_BAD_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1908_10583_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native._build, "LIB_PATH", str(tmp_path / "libfora.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _native.load()


def test_null_handles_and_counts_are_rejected_before_any_device_call(lib):
    """Entry points added for tuning, the walk index and the debug views check their
    arguments first: a null graph, key or output, or a negative count, is FORA_ERR_BAD_ARG
    with a message, and a zero count is a no-op (no device is touched)."""
    import ctypes
    v = ctypes.c_int64()
    d = ctypes.c_double()
    p = fora.Params.make()
    assert lib.fora_graph_tune(None, b"pipeline", 2) == fora.FORA_ERR_BAD_ARG
    assert lib.fora_graph_tuning(None, b"pipeline", ctypes.byref(v)) == fora.FORA_ERR_BAD_ARG
    assert lib.fora_index_build(None, ctypes.byref(p), None) == fora.FORA_ERR_BAD_ARG
    assert lib.fora_index_info(None, ctypes.byref(d), ctypes.byref(d), ctypes.byref(v)) == \
        fora.FORA_ERR_BAD_ARG
    assert lib.fora_index_export(None, None, None) == fora.FORA_ERR_BAD_ARG
    assert lib.fora_index_destroy(None) == fora.FORA_ERR_BAD_ARG
    assert lib.fora_threshold_debug(None, None, None, None, -1) == fora.FORA_ERR_BAD_ARG
    assert lib.fora_threshold_debug(None, None, None, None, 0) == fora.FORA_OK
    assert lib.fora_philox_debug(None, None, -1) == fora.FORA_ERR_BAD_ARG
    assert lib.fora_philox_debug(None, None, 0) == fora.FORA_OK
    assert lib.fora_last_error()


def test_workspace_bytes_counts_every_per_query_buffer(lib):
    """fora_workspace_bytes is host arithmetic over the same buffer sizes the workspace
    allocates and the serving lanes admit by.  Per query slot, counted by hand from the
    layout: residue, reserve (8 B each), walk tally (16 B), two frontier queues and the
    increments (8 B each) per node; two hub-item lists (8 B per hub chunk); per-source
    state (alist 4, counters 16, prefixes 16, source 4, r_max 8, stats 64, stop flag 4,
    light-round flag 1, edge count 8, one byte per 1024-node tile); top-k scratch
    (4096 histogram bins of 4 B, 32 B select state, 8192 candidates of 12 B); features
    64, prediction 4, learned r_max 8; staged results 4096 x (4 + 8)."""
    import inputs
    rp, _ = inputs.rmat_csr(12, 8, 1)
    n = len(rp) - 1
    deg = (rp[1:] - rp[:-1]).astype(int)
    hub_chunks = int(sum((d + 255) // 256 for d in deg if d > 256))
    per = (56 * n + 2 * 8 * hub_chunks + (4 + 16 + 16 + 4 + 8 + 64 + 4 + 1 + 8 + (n + 1023) // 1024)
           + (4096 * 4 + 32 + 8192 * 12) + (64 + 4 + 8) + 4096 * 12)
    b = [fora.workspace_bytes(rp, s) for s in (1, 2, 3, 64)]
    assert b[1] - b[0] == per and b[2] - b[1] == per
    assert b[3] == b[0] + 63 * per
    assert b[0] > per  # plus the fixed part (scan buffers, counters, loop state)
    with pytest.raises(fora.FORAError):
        fora.workspace_bytes(rp, 0)
    with pytest.raises(fora.FORAError):
        fora.workspace_bytes(rp[::-1].copy(), 1)


def test_fail_alloc_hook_arguments(lib):
    assert lib.fora_debug_fail_alloc(-1) == fora.FORA_ERR_BAD_ARG
    assert lib.fora_debug_fail_alloc(0) == fora.FORA_OK


def test_debug_build_has_index_checks_and_the_normal_build_not(lib):
    """FORA_DEBUG builds (device index checks, FORA_ERR_BOUNDS) are a separate library;
    fora_debug_checks says which one is loaded (host only, no device call)."""
    import ctypes
    assert lib.fora_debug_checks() == 0
    dbg = ctypes.CDLL(fbuild.build(debug=True))
    assert dbg.fora_debug_checks() == 1
    assert fora.header_functions() and all(hasattr(dbg, n) for n in fora.header_functions())


def _hot_reference(col, n, slots=128, min_indeg=64):
    """The hot-node rule written out with numpy: in-degree >= 64 and above the in-degree of
    the (slots+1)-th largest, ascending ids."""
    import numpy as np
    indeg = np.bincount(np.asarray(col, dtype=np.int64), minlength=n)
    cut = min_indeg
    if n > slots:
        cut = max(cut, int(np.sort(indeg)[n - slots - 1]) + 1)
    return np.flatnonzero(indeg >= cut)


def test_hot_nodes_of_the_push_follow_the_in_degree_rule(lib):
    """The nodes the spread sums per block (host arithmetic, no device): the rule against a
    numpy restatement on R-MAT graphs, a star, ties at the cut and graphs without hubs."""
    import numpy as np
    import inputs
    for scale, deg, seed in [(14, 8, 1), (12, 16, 5), (16, 4, 9)]:
        rp, col = inputs.rmat_csr(scale, deg, seed)
        got = fora.hot_nodes(rp, col)
        want = _hot_reference(col, len(rp) - 1)
        np.testing.assert_array_equal(got, want)
        assert 0 < len(got) <= 128
    # a star: every leaf points at the hub (in-degree 300), the hub at leaf 1
    n = 301
    col = np.concatenate([[1], np.zeros(n - 1, dtype=np.int32)]).astype(np.int32)
    rp = np.arange(n + 1, dtype=np.int64)
    np.testing.assert_array_equal(fora.hot_nodes(rp, col), [0])
    # 200 nodes tied at in-degree 100 (more than 128): all left out
    n = 200
    col = np.tile(np.arange(n, dtype=np.int32), 100)
    rp = np.arange(0, 100 * n + 1, 100, dtype=np.int64)
    assert len(fora.hot_nodes(rp, col)) == 0
    # 100 of 200 nodes tied at in-degree 100 (fewer than 128), the rest at 0: all 100 kept
    col = np.tile(np.arange(100, dtype=np.int32), 100)
    rp = np.arange(0, len(col) + 1, 50, dtype=np.int64)  # 200 rows of 50 edges
    np.testing.assert_array_equal(fora.hot_nodes(rp, col), np.arange(100))
    # no node reaches in-degree 64
    rp, col = np.arange(11, dtype=np.int64), np.arange(1, 11, dtype=np.int32) % 10
    assert len(fora.hot_nodes(rp, col)) == 0
    # bad arguments
    import ctypes
    c = ctypes.c_int32()
    assert lib.fora_hot_nodes(0, None, None, None, 0, ctypes.byref(c)) == fora.FORA_ERR_BAD_ARG
    bad = np.array([0, 5], dtype=np.int32)
    rp2 = np.array([0, 1, 2], dtype=np.int64)
    assert lib.fora_hot_nodes(2, rp2.ctypes.data, bad.ctypes.data, None, 0,
                              ctypes.byref(c)) == fora.FORA_ERR_BAD_ARG

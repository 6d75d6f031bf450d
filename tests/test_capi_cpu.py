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

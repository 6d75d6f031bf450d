"""fora_topk_noalloc (the top-k select with its scratch in a fixed device array, for
callers that cannot call cudaMalloc/cudaFree) against fora_topk, which allocates its
scratch per call.  Collected last on purpose: it runs after every other test, and
also passes alone in a fresh process.  Needs a GPU.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1908_10583_gb300 as fora  # noqa: E402
from paper_1908_10583_gb300 import build as fbuild  # noqa: E402


def _noalloc_topk(L, est, k):
    nrows, n = est.shape
    ids = torch.full((nrows, k), -1, dtype=torch.int32, device="cuda")
    vals = torch.full((nrows, k), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.fora_topk_noalloc(est.data_ptr(), n, nrows, k, ids.data_ptr(), vals.data_ptr(), stream)
    assert rc == fora.FORA_OK, L.fora_last_error()
    return ids, vals


def test_noalloc_topk_matches_the_allocating_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fbuild.build()
    L = fora.load()
    rng = np.random.default_rng(2024)
    # two calls in a row with different shapes: the second reuses the array the first
    # left behind, so a missing reset of the shared scratch would show here
    for n, nrows, k in [(300_000, 9, 500), (70_001, 3, 4096)]:
        est = rng.integers(0, 64, size=(nrows, n)) / 128.0  # heavy ties: ids decide
        est[:, ::5] = rng.random((nrows, len(range(0, n, 5))))
        est_t = torch.from_numpy(est).cuda()
        ids_a, vals_a = fora.topk(est_t, k)
        ids_b, vals_b = _noalloc_topk(L, est_t, k)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids_b.cpu().numpy(), ids_a.cpu().numpy())
        np.testing.assert_array_equal(vals_b.cpu().numpy(), vals_a.cpu().numpy())


def test_noalloc_topk_rejects_more_rows_than_its_array_holds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fbuild.build()
    L = fora.load()
    est = torch.zeros((10, 1000), dtype=torch.float64, device="cuda")
    out_i = torch.zeros((10, 5), dtype=torch.int32, device="cuda")
    out_v = torch.zeros((10, 5), dtype=torch.float64, device="cuda")
    rc = L.fora_topk_noalloc(est.data_ptr(), 1000, 10, 5, out_i.data_ptr(), out_v.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    assert rc == fora.FORA_ERR_BAD_ARG
    assert b"9 rows" in L.fora_last_error()

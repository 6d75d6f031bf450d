"""Serving with continuous batching (needs a GPU): every result is the same alone and in
the mix, within the push tolerance, and batches overlap on the device."""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1908_10583_gb300 as fora  # noqa: E402
from paper_1908_10583_gb300 import build as fbuild  # noqa: E402

ATOL_PUSH = 1e-12


def test_results_are_the_same_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fbuild.build()
    graphs = [fora.Graph(*inputs.rmat_csr(14, 8, 1)), fora.Graph(*inputs.rmat_csr(16, 16, 5))]
    server = fora.Server(graphs, lanes_per_graph=2, max_batch=16,
                         memory_budget_bytes=2 << 30, batch_window_ms=2.0)
    rng = np.random.default_rng(9)
    reqs = []
    for i in range(64):
        gi = int(rng.integers(0, 2))
        p = fora.Params.make(eps=float(rng.choice([0.5, 0.3])), k=int(rng.choice([50, 200])),
                             seed=77)
        src = int(rng.integers(0, graphs[gi].n))
        reqs.append((gi, src, p, server.submit(gi, src, p)))
    results = [(gi, src, p, *server.wait(t, p.k)) for gi, src, p, t in reqs]
    st = server.stats()
    assert st["completed"] == 64
    assert st["batches"] < 64                     # requests shared batches
    assert st["max_concurrent_lanes"] >= 2        # batches overlapped on the device
    assert max(info.batch_size for *_, info in results) > 1
    for gi, src, p, ids, vals, info in results:
        ids1, vals1, st1 = graphs[gi].ssppr(src, p)   # the same query alone
        np.testing.assert_allclose(vals, vals1, rtol=0, atol=ATOL_PUSH)
        assert info.stats.walks == st1.walks
        differ = ids != ids1
        if differ.any():  # only between estimates that are equal within the tolerance
            assert np.all(np.abs(vals[differ] - vals1[differ]) <= 2 * ATOL_PUSH)
    server.close()

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


def test_arrivals_join_running_batches_and_match_the_query_alone():
    """Requests arriving while a lane's batch is in its push rounds take free slots of that
    batch between two rounds: such a request finishes with a batch that had already started
    before it arrived (instead of waiting for the next one), and its result is the same as
    the query alone (values within the push tolerance, same walk count)."""
    import time
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fbuild.build()
    g = fora.Graph(*inputs.rmat_csr(20, 16, 2))
    server = fora.Server([g], lanes_per_graph=1, max_batch=64, memory_budget_bytes=16 << 30,
                         batch_window_ms=0.0, admit_during_push=True)
    p = fora.Params.make(eps=0.5, k=50, seed=21)
    src = inputs.uniform_sources(g.n, 120, 2024)
    tickets = []
    for s in src:  # arrivals spread over about 60 ms, several batches' push rounds
        tickets.append(server.submit(0, int(s), p))
        time.sleep(0.0005)
    results = [server.wait(t, 50) for t in tickets]
    st = server.stats()
    assert st["completed"] == len(src) and st["joined"] >= 1
    infos = [info for _, _, info in results]
    joined = [i for i, info in enumerate(infos) if info.joined]
    assert len(joined) == st["joined"]
    for j in joined:  # it finished with a batch that had started before it was submitted
        J = infos[j]
        assert any(R.start_ms < J.submit_ms and R.end_ms == J.end_ms and not R.joined
                   for R in infos)
    for s, (ids, vals, info) in zip(src, results):
        ids1, vals1, st1 = g.ssppr(int(s), p)
        np.testing.assert_allclose(vals, vals1, rtol=0, atol=ATOL_PUSH)
        assert info.stats.walks == st1.walks and info.stats.pushes == st1.pushes
    server.close()
    g.close()

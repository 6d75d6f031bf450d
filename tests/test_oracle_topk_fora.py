"""Pins for the oracle's top-k FORA (Alg. 5), CPU only."""
import numpy as np
import pytest

import inputs
import oracle
from oracle import exact


@pytest.mark.parametrize("k", [10, 50])
def test_topk_fora_meets_def2(k):
    """Def. 2 against power iteration: pi_hat(v_i) >= (1 - eps) pi(v_i) and
    pi(v_i) >= (1 - eps) pi(v*_i) for every i with pi(v*_i) > 1/n."""
    rp, col = inputs.rmat_csr(12, 8, 6)
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 5, 303)
    truth = exact.power_iteration(rp, col, 0.2, sources)
    eps = 0.5
    for i, s in enumerate(sources):
        q = oracle.topk_fora(rp, col, s, k, eps=eps)
        true_sorted = np.sort(truth[i])[::-1]
        for j, v in enumerate(q.ids):
            if true_sorted[j] > 1.0 / n:
                assert q.vals[j] >= (1 - eps) * truth[i][v]
                assert truth[i][v] >= (1 - eps) * true_sorted[j]
        # Lemma (topk-delta): it stops with delta <= pi(s, v*_k) (except w.p. <= n p_f'/8)
        assert q.delta <= true_sorted[k - 1]
        assert 1 <= q.iterations <= int(np.ceil(np.log2(n / k))) + 1


def test_topk_fora_stops_early_for_a_concentrated_source():
    """A source whose top-k mass is large stops at delta = 1/k after one round: the k-th
    estimate of a 2-cycle with alpha = 1/2 is 1/3 >= (1 + eps)/k for k = 2."""
    rp, col = inputs.csr_from_edges(2, [(0, 1), (1, 0)])
    q = oracle.topk_fora(rp, col, 0, 2, alpha=0.5, eps=0.5)
    assert q.iterations == 1 and q.delta == 0.5
    np.testing.assert_allclose(q.vals, [2 / 3, 1 / 3], atol=0.1)


def test_topk_fora_last_round_is_the_whole_graph_query():
    """k = n: a single round with delta = 1/n, eps/2 and p_f/n: the plain query's top-k."""
    rp, col = inputs.rmat_csr(8, 4, 2)
    n = len(rp) - 1
    q = oracle.topk_fora(rp, col, 3, n, eps=0.5, seed=99)
    assert q.iterations == 1 and q.delta == 1.0 / n
    w = oracle.ssppr(rp, col, 3, eps=0.25, delta=1.0 / n, pf=1.0 / n / n, k=n, seed=99)
    np.testing.assert_array_equal(q.ids, w.ids)
    np.testing.assert_array_equal(q.vals, w.vals)

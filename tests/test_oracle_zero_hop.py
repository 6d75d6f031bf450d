"""Pins for the oracle's zero-hop pruned walk phase (Section 4.1), CPU only."""
import numpy as np
import pytest

import inputs
import oracle
from oracle import exact
from test_oracle_push import random_graph
from test_oracle_walks import chi2_pvalue


@pytest.mark.parametrize("seed,alpha", [(31, 0.2), (32, 0.5)])
def test_forced_first_move_end_distribution(seed, alpha):
    """A pruned walk from v first moves to a uniform out-neighbour, so it ends at t with
    probability pi_1(v, t) / (1 - alpha) = (pi(v, t) - alpha [t = v]) / (1 - alpha)."""
    n = 12
    rp, col = random_graph(n, 3, seed)
    v = 5
    pi = exact.dense_ppr(rp, col, alpha, [v])[0]
    want = pi.copy()
    want[v] -= alpha
    want /= 1 - alpha
    N = 200_000
    residue = np.zeros(n)
    residue[v] = 1.0 / (1 - alpha)  # r'(v) = 1, so omega_v = N with C = N
    count, acc, st = oracle.walk_phase_zero_hop(rp, col, 0, alpha, float(N), 77, residue)
    assert st.walks == N == count.sum()
    assert chi2_pvalue(count.astype(float), N * want) > 1e-6
    # every walk makes the forced move, then (1 - alpha) / alpha more on average
    assert st.walk_steps / N == pytest.approx(1 + (1 - alpha) / alpha, rel=0.02)


def test_zero_hop_estimator_is_unbiased():
    """pi = reserve + alpha r + sum_v r'(v) E[X_v] (Section 4.1): average over seeds."""
    n = 20
    rp, col = random_graph(n, 3, 21)
    alpha, s = 0.2, 3
    pi = exact.dense_ppr(rp, col, alpha, [s])[0]
    res, r, _ = oracle.forward_push(rp, col, s, alpha, 0.02)
    ests = []
    for seed in range(300):
        _, acc, _ = oracle.walk_phase_zero_hop(rp, col, s, alpha, 200.0, seed, r)
        ests.append(oracle.estimate_zero_hop(res, r, acc, alpha))
    ests = np.array(ests)
    mean, sem = ests.mean(0), ests.std(0, ddof=1) / np.sqrt(len(ests))
    assert np.all(np.abs(mean - pi) <= 5 * sem + 1e-12)


def test_zero_hop_query_is_eps_accurate_with_fewer_walks():
    rp, col = inputs.rmat_csr(12, 8, 6)
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 6, 101)
    truth = exact.power_iteration(rp, col, 0.2, sources)
    for i, s in enumerate(sources):
        q = oracle.ssppr(rp, col, s, eps=0.5, k=50, zero_hop=True)
        q0 = oracle.ssppr(rp, col, s, eps=0.5, k=50)
        big = truth[i] >= 1.0 / n
        rel = np.abs(q.est[big] - truth[i][big]) / truth[i][big]
        assert rel.max() <= 0.5
        np.testing.assert_array_equal(q.reserve, q0.reserve)  # same push
        # omega_v = ceil((1 - alpha) r(v) C): about (1 - alpha) of the walks
        assert 0.78 * q0.walk.walks <= q.walk.walks <= 0.82 * q0.walk.walks + q.walk.residual_nodes

"""Pins for the oracle's random-walk phase, estimate and top-k (CPU only)."""
import numpy as np
import pytest
from scipy import stats

import inputs
import oracle
from oracle import exact
from test_oracle_push import random_graph

TWO63 = float(2**63)


def chi2_pvalue(observed, expected):
    mask = expected > 0
    assert observed[~mask].sum() == 0, "walk ended where the exact PPR is zero"
    chi2 = ((observed[mask] - expected[mask]) ** 2 / expected[mask]).sum()
    return stats.chi2.sf(chi2, df=mask.sum() - 1)


@pytest.mark.parametrize("seed,alpha", [(11, 0.2), (12, 0.5), (13, 0.05)])
def test_walk_end_distribution_is_ppr(seed, alpha):
    """Section 2.1: a walk from v stops at t with probability pi(v, t).
    One residual node, N walks: counts ~ Multinomial(N, pi(v, .))."""
    n = 12
    rp, col = random_graph(n, 3, seed)
    v = 4
    pi = exact.dense_ppr(rp, col, alpha, [v])[0]
    N = 200_000
    residue = np.zeros(n)
    residue[v] = 1.0
    count, acc, st = oracle.walk_phase(rp, col, 0, alpha, float(N), 99, residue)
    assert st.walks == N and count.sum() == N
    assert chi2_pvalue(count.astype(float), N * pi) > 1e-6
    # mean walk length (1 - alpha) / alpha
    assert st.walk_steps / N == pytest.approx((1 - alpha) / alpha, rel=0.02)


def test_neighbour_choice_is_uniform_on_odd_degree():
    """Star 0 -> {1..7}, leaves -> 0, alpha = 1/2: by symmetry the leaves share
    pi(0, leaf) equally; a biased index draw (e.g. modulo) would break the symmetry."""
    rp, col = inputs.csr_from_edges(8, [(0, i) for i in range(1, 8)] + [(i, 0) for i in range(1, 8)])
    pi = exact.dense_ppr(rp, col, 0.5, [0])[0]
    assert np.allclose(pi[1:], pi[1])
    residue = np.zeros(8)
    residue[0] = 1.0
    N = 300_000
    count, _, _ = oracle.walk_phase(rp, col, 0, 0.5, float(N), 3, residue)
    assert chi2_pvalue(count.astype(float), N * pi) > 1e-6


def test_multiplicity_and_self_loops_in_walks():
    """0 -> {0, 1, 1}: the walk stays with prob 1/3 and moves to 1 with 2/3."""
    rp, col = inputs.csr_from_edges(2, [(0, 0), (0, 1), (0, 1), (1, 0)])
    pi = exact.dense_ppr(rp, col, 0.3, [0])[0]
    residue = np.array([1.0, 0.0])
    N = 200_000
    count, _, _ = oracle.walk_phase(rp, col, 0, 0.3, float(N), 5, residue)
    assert chi2_pvalue(count.astype(float), N * pi) > 1e-6


def test_walk_counts_and_weights_conserve():
    """omega_v = ceil(r(v) C) walks per residual node; the fixed-point weights of all walks
    sum exactly to sum_v omega_v W_v, which is r_sum up to half a unit per walk."""
    rp, col = inputs.rmat_csr(10, 8, 3)
    n = len(rp) - 1
    rmax = 1e-3
    res, r, pst = oracle.forward_push(rp, col, 9, 0.2, rmax)
    C = 3.0e4
    count, acc, st = oracle.walk_phase(rp, col, 9, 0.2, C, 1234, r)
    omega = np.ceil(r[r > 0] * C)
    assert st.walks == omega.sum() == count.sum()
    assert st.residual_nodes == (r > 0).sum()
    total = sum(int(a) for a in acc)
    assert abs(total / TWO63 - r.sum()) <= st.walks / TWO63 + 1e-15


def test_walk_phase_is_deterministic_and_seeded():
    rp, col = inputs.rmat_csr(10, 8, 3)
    _, r, _ = oracle.forward_push(rp, col, 2, 0.2, 1e-3)
    a = oracle.walk_phase(rp, col, 2, 0.2, 1e4, 7, r)
    b = oracle.walk_phase(rp, col, 2, 0.2, 1e4, 7, r)
    c = oracle.walk_phase(rp, col, 2, 0.2, 1e4, 8, r)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert (a[0] != c[0]).any()


def test_estimator_is_unbiased():
    """Eq. (connection)/(ss-exp): E[pi_hat(s, t)] = pi(s, t).  Average over seeds."""
    n = 20
    rp, col = random_graph(n, 3, 21)
    alpha, s = 0.2, 3
    pi = exact.dense_ppr(rp, col, alpha, [s])[0]
    res, r, _ = oracle.forward_push(rp, col, s, alpha, 0.02)
    C = 200.0
    ests = []
    for seed in range(300):
        _, acc, _ = oracle.walk_phase(rp, col, s, alpha, C, seed, r)
        ests.append(oracle.estimate(res, acc))
    ests = np.array(ests)
    mean, sem = ests.mean(0), ests.std(0, ddof=1) / np.sqrt(len(ests))
    assert np.all(np.abs(mean - pi) <= 5 * sem + 1e-12)


def test_monte_carlo_special_case():
    """r_max >= 1: no push, every walk starts at s with weight 1/ceil(C): pi_hat = count/ceil(C)."""
    rp, col = inputs.rmat_csr(9, 8, 4)
    n = len(rp) - 1
    q = oracle.ssppr(rp, col, 5, rmax=1.0, k=10)
    assert q.push.rounds == 0 and q.walk.residual_nodes == 1
    N = q.walk.walks
    w = round(TWO63 / N)
    np.testing.assert_array_equal(q.acc, q.count.astype(np.uint64) * np.uint64(w))
    np.testing.assert_allclose(q.est, q.count / N, rtol=1e-12, atol=0)


def test_estimate_fixed_point_scale():
    est = oracle.estimate(np.array([0.25, 0.0, 1e-3]),
                          np.array([2**62, 2**63, 0], dtype=np.uint64))
    np.testing.assert_array_equal(est, [0.75, 1.0, 1e-3])


@pytest.mark.parametrize("seed", range(4))
def test_topk_against_brute_force_with_ties(seed):
    rng = np.random.default_rng(seed)
    n = 3000
    est = rng.integers(0, 40, size=n) / 40.0  # many ties
    k = 57
    ids, vals = oracle.topk(est, k)
    order = np.lexsort((np.arange(n), -est))[:k]
    np.testing.assert_array_equal(ids, order)
    np.testing.assert_array_equal(vals, est[order])


def test_whole_query_is_eps_accurate():
    """Lemma (layerppr-conc): |pi_hat - pi| <= eps pi for every t with pi(s,t) >= delta,
    except with probability p_f per source (1/n here: expect no failure on 6 sources)."""
    rp, col = inputs.rmat_csr(12, 8, 6)
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 6, 101)
    truth = exact.power_iteration(rp, col, 0.2, sources)
    eps = 0.5
    for i, s in enumerate(sources):
        q = oracle.ssppr(rp, col, s, eps=eps, k=50)
        big = truth[i] >= 1.0 / n
        rel = np.abs(q.est[big] - truth[i][big]) / truth[i][big]
        assert rel.max() <= eps, (s, rel.max())
        # the estimate carries the reserve exactly and only adds walk weight
        assert np.all(q.est >= q.reserve)
        # Def. 2 (top-k accuracy) with the same guarantee
        true_sorted = np.sort(truth[i])[::-1]
        for j, v in enumerate(q.ids):
            if true_sorted[j] > 1.0 / n:
                assert q.est[v] >= (1 - eps) * truth[i][v]
                assert truth[i][v] >= (1 - eps) * true_sorted[j]

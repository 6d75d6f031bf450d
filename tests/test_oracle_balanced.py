"""Pins for the oracle's balanced Forward Push (Section 4.2, Alg. 3), CPU only.

Reading: the threshold theta starts at 1 and halves whenever no node is above it; before
each round the push stops once its cost so far, FC = cost_edge * edge pushes + cost_push *
node pushes, reaches the estimated walk cost (r_sum * C') * cost_walk."""
import numpy as np
import pytest

import inputs
import oracle
from oracle import exact
from tests.test_oracle_push import random_graph


def test_two_cycle_by_hand():
    """0 <-> 1 (d = 1), alpha = 0.2, C' = 1, cost_walk = 1, cost_push = 0.
    theta = 1: r(0) = 1 is not above 1 * 1, so theta = 1/2; round 1 pushes {0}:
    reserve(0) = 0.2, r(1) = 0.8, FC = cost_edge, walk cost (1 - 0.2) * 1 * 1 = 0.8.
    cost_edge = 0.5: FC = 0.5 < 0.8, round 2 pushes {1} (0.8 > 1/2): reserve(1) = 0.16,
    r(0) = 0.64; FC = 1.0 >= 0.64: stop.
    cost_edge = 0.3: after round 2 FC = 0.6 < 0.64, round 3 pushes {0} (0.64 > 1/2):
    reserve(0) = 0.328, r(1) = 0.512; FC = 0.9 >= 0.512: stop."""
    rp, col = inputs.csr_from_edges(2, [(0, 1), (1, 0)])
    res, r, st, theta = oracle.forward_push_balanced(rp, col, 0, 0.2, 1.0, 0.5, 0.0, 1.0)
    assert (st.rounds, st.pushes, st.edge_pushes, theta) == (2, 2, 2, 0.5)
    np.testing.assert_allclose(res, [0.2, 0.16], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r, [0.64, 0.0], rtol=0, atol=1e-15)
    res, r, st, theta = oracle.forward_push_balanced(rp, col, 0, 0.2, 1.0, 0.3, 0.0, 1.0)
    assert (st.rounds, st.pushes, theta) == (3, 3, 0.5)
    np.testing.assert_allclose(res, [0.328, 0.16], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r, [0.0, 0.512], rtol=0, atol=1e-15)


def test_threshold_halves_when_nobody_is_above_it():
    """Star 0 -> {1, 2, 3, 4}, leaves back to 0, alpha = 1/2, cost_push = 1, no edge
    cost, cost_walk = 4, C' = 1: theta goes 1 -> 1/2 -> 1/4 -> 1/8 before r(0) = 1 is above
    theta * 4; round 1 pushes {0} (FC = 1 < (1 - 1/2) * 4 = 2), each leaf gets 1/8 =
    theta * 1, not above it, so theta halves to 1/16 and round 2 pushes the four leaves:
    FC = 5 >= (1 - 3/4) * 4 = 1 stops the push with r(0) = 4 * (1/2) (1/8) = 1/4."""
    rp, col = inputs.csr_from_edges(5, [(0, 1), (0, 2), (0, 3), (0, 4),
                                        (1, 0), (2, 0), (3, 0), (4, 0)])
    res, r, st, theta = oracle.forward_push_balanced(rp, col, 0, 0.5, 1.0, 0.0, 1.0, 4.0)
    assert st.rounds == 2 and st.pushes == 5 and theta == 1.0 / 16
    np.testing.assert_allclose(res, [0.5, 1 / 16, 1 / 16, 1 / 16, 1 / 16], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r, [0.25, 0, 0, 0, 0], rtol=0, atol=1e-15)


def test_free_walks_mean_no_push():
    """cost_walk = 0: the estimated walk cost is 0 and FC = 0 already meets it, so
    nothing is pushed (FORA reduces to Monte-Carlo)."""
    rp, col = random_graph(20, 3, 1)
    res, r, st, theta = oracle.forward_push_balanced(rp, col, 4, 0.2, 1e4, 1.0, 1.0, 0.0)
    assert st.pushes == 0 and theta == 1.0
    assert not res.any() and r[4] == 1.0 and r.sum() == 1.0


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("cost_walk", [1e-4, 1e-2, 1.0, 100.0])
def test_invariant_against_dense_solve(seed, cost_walk):
    """Wherever the cost rule stops it, the push leaves Eq. (layerppr) intact:
    pi(s, t) = reserve(t) + sum_v r(v) pi(v, t), with the exact PPR of a dense solve; the
    mass reserve + residue is 1 and r_sum at the stop is consistent with the rule."""
    rp, col = random_graph(24, 3, 100 + seed)
    n = len(rp) - 1
    s = seed % n
    C = 500.0
    res, r, st, theta = oracle.forward_push_balanced(rp, col, s, 0.2, C, 1.0, 0.5, cost_walk)
    P = exact.dense_ppr(rp, col, 0.2, range(n))
    np.testing.assert_allclose(res + r @ P, P[s], rtol=0, atol=1e-12)
    assert abs(res.sum() + r.sum() - 1.0) < 1e-13
    fc = 1.0 * st.edge_pushes + 0.5 * st.pushes
    assert fc >= r.sum() * C * cost_walk - 1e-9
    assert theta > 0 and np.log2(theta) == np.round(np.log2(theta))


def test_costlier_walks_mean_more_push():
    """A higher walk cost keeps the push going longer: more node pushes and a smaller
    residue sum left for the walks (the trade Alg. 3 balances)."""
    rp, col = inputs.rmat_csr(10, 6, 7)
    prev_pushes, prev_rsum = -1, 2.0
    for cw in (1e-7, 1e-6, 1e-5, 1e-4):
        _, r, st, _ = oracle.forward_push_balanced(rp, col, 3, 0.2, 1e6, 1.0, 1.0, cw)
        assert st.pushes >= prev_pushes and r.sum() <= prev_rsum + 1e-15
        prev_pushes, prev_rsum = st.pushes, r.sum()
    assert prev_pushes > 0

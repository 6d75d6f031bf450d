"""Pins for the ground truth (dense solve, power iteration) and the input generator."""
import numpy as np
import pytest

import inputs
from oracle import exact
from test_oracle_push import random_graph


def test_directed_cycle_closed_form():
    """Cycle 0 -> 1 -> ... -> L-1 -> 0: the walk from 0 stops after i moves with
    probability alpha (1-alpha)^i, so pi(0, i) = alpha (1-alpha)^i / (1 - (1-alpha)^L)."""
    L, alpha = 7, 0.2
    rp, col = inputs.csr_from_edges(L, [(i, (i + 1) % L) for i in range(L)])
    want = alpha * (1 - alpha) ** np.arange(L) / (1 - (1 - alpha) ** L)
    np.testing.assert_allclose(exact.dense_ppr(rp, col, alpha, [0])[0], want, rtol=1e-13)
    np.testing.assert_allclose(exact.power_iteration(rp, col, alpha, [0])[0], want, rtol=1e-13)


def test_complete_graph_with_self_loops_closed_form():
    """Every node links to all n nodes: pi(s, t) = alpha [s = t] + (1 - alpha) / n."""
    n, alpha = 9, 0.3
    rp, col = inputs.csr_from_edges(n, [(i, j) for i in range(n) for j in range(n)])
    want = np.full(n, (1 - alpha) / n)
    want[2] += alpha
    np.testing.assert_allclose(exact.dense_ppr(rp, col, alpha, [2])[0], want, rtol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_power_iteration_matches_dense_solve(seed):
    rp, col = random_graph(60, 4, seed)
    src = [0, 7, 31]
    np.testing.assert_allclose(exact.power_iteration(rp, col, 0.2, src),
                               exact.dense_ppr(rp, col, 0.2, src), rtol=0, atol=1e-14)


def test_ppr_rows_are_distributions():
    rp, col = random_graph(30, 3, 9)
    Pi = exact.dense_ppr(rp, col, 0.2, list(range(30)))
    np.testing.assert_allclose(Pi.sum(1), 1.0, atol=1e-13)
    assert (Pi >= -1e-16).all() and (np.diag(Pi) >= 0.2).all()


def test_rmat_generator_shape_and_determinism():
    rp, col = inputs.rmat_csr(12, 8, 1)
    n = len(rp) - 1
    deg = np.diff(rp)
    assert n == 4096 and (deg >= 1).all() and rp[0] == 0
    assert col.min() >= 0 and col.max() < n
    raw = 8 * n
    assert rp[-1] == raw + 0 + (rp[-1] - raw) and rp[-1] >= raw
    for v in range(0, n, 97):  # rows sorted ascending
        row = col[rp[v]:rp[v + 1]]
        assert (np.diff(row) >= 0).all()
    rp1, col1 = inputs.rmat_csr(12, 8, 1, nthreads=1)
    np.testing.assert_array_equal(rp, rp1)
    np.testing.assert_array_equal(col, col1)
    rp2, _ = inputs.rmat_csr(12, 8, 2)
    assert (rp2 != rp).any()
    # skew: R-MAT with a = 0.57 gives a heavy-tailed out-degree
    assert deg.max() > 20 * deg.mean()


def test_uniform_sources():
    s = inputs.uniform_sources(1000, 20000, 101)
    assert s.min() >= 0 and s.max() < 1000
    counts = np.bincount(s, minlength=1000)
    assert counts.min() > 0 and abs(counts.mean() - 20) < 1e-9
    np.testing.assert_array_equal(s, inputs.uniform_sources(1000, 20000, 101))

"""Pins for the oracle's Forward Push (Alg. 1, synchronous rounds), CPU only."""
import numpy as np
import pytest

import inputs
import oracle
from oracle import exact


def random_graph(n, avg_deg, seed, self_loops=True):
    """Small random directed multigraph with d_out >= 1 everywhere."""
    rng = np.random.default_rng(seed)
    edges = []
    for v in range(n):
        d = 1 + rng.poisson(avg_deg - 1)
        for u in rng.integers(0, n, size=d):
            if self_loops or u != v:
                edges.append((v, int(u)))
        if not any(e[0] == v for e in edges[-d:]):
            edges.append((v, (v + 1) % n))
    return inputs.csr_from_edges(n, edges)


def test_two_cycle_by_hand():
    """0 <-> 1, alpha = 1/2, r_max = 0.2: residue halves and hops each round;
    rounds: {0}, {1}, {0}; then r(1) = 1/8 <= 0.2 stops the push."""
    rp, col = inputs.csr_from_edges(2, [(0, 1), (1, 0)])
    res, r, st = oracle.forward_push(rp, col, 0, 0.5, 0.2)
    assert st.rounds == 3 and st.pushes == 3 and st.edge_pushes == 3
    np.testing.assert_array_equal(res, [0.625, 0.25])
    np.testing.assert_array_equal(r, [0.0, 0.125])


def test_triangle_rounds_are_synchronous_by_hand():
    """0->1, 0->2, 1->2, 2->0 with alpha = 1/2, r_max = 0.1.
    round 1: F={0}: res0=1/2, r1=r2=1/4.
    round 2: F={1,2}: both reserves take 1/8 and both residues go to 0 first; then 1->2 adds
             1/8 to r2 (it waits for round 3) and 2->0 adds 1/8 to r0.
    round 3: F={2} (r0 = 1/8 <= 0.1*2): res2 = 1/8 + 1/16, r0 = 1/8 + 1/16 = 3/16 <= 0.2.
    A sequential push that let node 2 take 1's increment within round 2 would end elsewhere."""
    rp, col = inputs.csr_from_edges(3, [(0, 1), (0, 2), (1, 2), (2, 0)])
    res, r, st = oracle.forward_push(rp, col, 0, 0.5, 0.1)
    assert st.rounds == 3 and st.pushes == 4
    np.testing.assert_array_equal(res, [0.5, 0.125, 0.1875])
    np.testing.assert_array_equal(r, [0.1875, 0.0, 0.0])


def test_multiplicity_counts():
    """Parallel edges: 0 -> {1, 1, 2}: node 1 gets two shares of (1-alpha)/3; then
    r(1) = 1/2 <= 0.3 * 2 and r(2) = 1/4 <= 0.3 * 1 end the push after one round."""
    rp, col = inputs.csr_from_edges(3, [(0, 1), (0, 1), (0, 2), (1, 0), (1, 0), (2, 0)])
    res, r, st = oracle.forward_push(rp, col, 0, 0.25, 0.3)
    assert st.rounds == 1
    np.testing.assert_allclose(r, [0.0, 2 * 0.75 / 3, 0.75 / 3], rtol=0, atol=1e-16)
    assert res[0] == 0.25


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("rmax", [0.3, 0.05, 1e-3, 1e-5])
def test_invariant_against_dense_solve(seed, rmax):
    """Eq. (layerppr): pi(s,t) = reserve(t) + sum_v r(v) pi(v,t), exact pi by LU."""
    n = 40
    rp, col = random_graph(n, 3, seed)
    alpha = 0.2
    Pi = exact.dense_ppr(rp, col, alpha, list(range(n)))
    s = seed % n
    res, r, st = oracle.forward_push(rp, col, s, alpha, rmax)
    np.testing.assert_allclose(res + r @ Pi, Pi[s], rtol=0, atol=1e-13)
    # mass: every push turns r(v) into alpha r(v) reserve + (1-alpha) r(v) residue
    assert res.sum() + r.sum() == pytest.approx(1.0, abs=1e-13)
    # termination condition of Alg. 1: r(v) <= r_max d_out(v) for every v
    assert np.all(r <= rmax * np.diff(rp))
    # O(1/r_max) bound of Section 2.2: each push of v moves more than alpha r_max d(v)
    assert st.edge_pushes < 1.0 / (alpha * rmax)
    assert st.rsum == pytest.approx(r.sum(), abs=1e-15)


def test_no_push_when_rmax_at_least_one():
    """r(s)/d(s) = 1/d(s) <= r_max: Alg. 1 does nothing and FORA reduces to Monte-Carlo."""
    rp, col = random_graph(30, 3, 1)
    res, r, st = oracle.forward_push(rp, col, 5, 0.2, 1.0)
    assert st.rounds == 0
    assert not res.any()
    assert r[5] == 1.0 and r.sum() == 1.0


def test_tiny_rmax_converges_to_exact_ppr():
    rp, col = random_graph(50, 4, 7)
    Pi = exact.dense_ppr(rp, col, 0.2, [3])[0]
    res, r, st = oracle.forward_push(rp, col, 3, 0.2, 1e-12)
    assert np.abs(res - Pi).max() <= r.sum() + 1e-15
    assert r.sum() < 1e-9


def test_rejects_dangling_and_bad_args():
    rp, col = inputs.csr_from_edges(3, [(0, 1), (1, 0)])  # node 2 has no out-edge
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward_push(rp, col, 0, 0.2, 0.1)
    assert e.value.code == -2
    rp, col = inputs.csr_from_edges(2, [(0, 1), (1, 0)])
    with pytest.raises(oracle.OracleError):
        oracle.forward_push(rp, col, 5, 0.2, 0.1)
    with pytest.raises(oracle.OracleError):
        oracle.forward_push(rp, col, 0, 1.0, 0.1)


def test_rmat_push_invariants():
    """Invariants on an R-MAT graph at the rule's r_max (no dense solve at this size)."""
    rp, col = inputs.rmat_csr(12, 8, 5)
    n = len(rp) - 1
    rmax = oracle.rmax_rule(0.5, 1.0 / n, 1.0 / n, rp[-1])
    res, r, st = oracle.forward_push(rp, col, 17, 0.2, rmax)
    assert res.sum() + r.sum() == pytest.approx(1.0, abs=1e-12)
    assert np.all(r <= rmax * np.diff(rp))
    assert st.rounds > 3 and st.edge_pushes < 1.0 / (0.2 * rmax)
    assert r.sum() <= rp[-1] * rmax  # r_sum <= m r_max (Section 3.2)

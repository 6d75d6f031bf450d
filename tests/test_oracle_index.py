"""Pins for the oracle's FORA+ walk index (Section 3.3) and its indexed walk phase (CPU).

The index holds, for every node v, the ends of omega_max(v) walks from v; a query that
needs omega_v <= omega_max(v) walks from v reads the first omega_v of them.  Pinned by:
the indexed phase equals the simulated walk phase exactly when the index walks use the
query's own Philox streams (same walks); omega_v <= omega_max(v) for every residue the
push leaves; the index size against the bound of Lemma (idx-size); the stored ends follow
the PPR distribution (chi-square against a dense solve).
"""
import numpy as np
import pytest
from scipy import stats

import inputs
import oracle
from oracle import exact


@pytest.fixture(scope="module")
def graph():
    rp, col = inputs.rmat_csr(10, 6, 21)
    return rp, col


def test_indexed_phase_equals_walk_phase_with_the_same_streams(graph):
    rp, col = graph
    n = len(rp) - 1
    s = 17
    C = oracle.walk_scale(0.5, 1.0 / n, 1.0 / n)
    rmax = oracle.rmax_rule(0.5, 1.0 / n, 1.0 / n, rp[-1])
    reserve, residue, _ = oracle.forward_push(rp, col, s, 0.2, rmax)
    off, dest = oracle.walk_index(rp, col, 0.2, C, rmax, seed=99, s_index=s)
    cnt_i, acc_i, st_i = oracle.walk_phase_indexed(n, C, residue, off, dest)
    cnt_w, acc_w, st_w = oracle.walk_phase(rp, col, s, 0.2, C, 99, residue)
    np.testing.assert_array_equal(cnt_i, cnt_w)
    np.testing.assert_array_equal(acc_i, acc_w)
    assert st_i.walks == st_w.walks and st_i.residual_nodes == st_w.residual_nodes
    assert st_i.walk_steps == 0


def test_push_residues_never_need_more_walks_than_the_index_holds(graph):
    rp, col = graph
    n = len(rp) - 1
    deg = np.diff(rp)
    for eps in (0.5, 0.2):
        C = oracle.walk_scale(eps, 1.0 / n, 1.0 / n)
        rmax = oracle.rmax_rule(eps, 1.0 / n, 1.0 / n, rp[-1])
        omega_max = np.ceil((rmax * deg) * C)
        for s in (0, 5, 300, n - 1):
            _, residue, _ = oracle.forward_push(rp, col, s, 0.2, rmax)
            omega = np.ceil(residue * C)
            assert np.all(omega <= omega_max)


def test_index_size_and_layout(graph):
    """Sum of omega_max(v) is at most n + r_max m C (each ceiling adds < 1), and with the
    rule's Case 1 r_max it is at most n + sqrt(m (2eps/3+2) log(2/p_f) / delta) / eps
    (Section 3.3); offsets are the prefix of omega_max, every end is a node id."""
    rp, col = graph
    n, m = len(rp) - 1, int(rp[-1])
    eps, delta, pf = 0.5, 1.0 / n, 1.0 / n
    C = oracle.walk_scale(eps, delta, pf)
    rmax = oracle.rmax_rule(eps, delta, pf, m)
    off, dest = oracle.walk_index(rp, col, 0.2, C, rmax, seed=3)
    deg = np.diff(rp)
    np.testing.assert_array_equal(np.diff(off), np.ceil((rmax * deg) * C).astype(np.int64))
    assert off[-1] <= n + rmax * m * C
    assert off[-1] <= n + np.sqrt(m * (2 * eps / 3 + 2) * np.log(2 / pf) / delta) / eps
    assert len(dest) == off[-1] and dest.min() >= 0 and dest.max() < n


def test_index_walk_ends_follow_ppr():
    """The stored ends of the walks from one node, pooled over many omega_max, are samples
    of pi(v, .) (Section 2.1): chi-square against the dense solve."""
    rp, col = inputs.rmat_csr(6, 4, 5)
    n = len(rp) - 1
    off, dest = oracle.walk_index(rp, col, 0.2, 4000.0, 1.0, seed=11)
    v = int(np.argmax(np.diff(off)))
    pi = exact.dense_ppr(rp, col, 0.2, [v])[0]
    ends = dest[off[v]:off[v + 1]]
    assert len(ends) >= 2000
    obs = np.bincount(ends, minlength=n).astype(np.float64)
    exp_ = pi * len(ends)
    keep = exp_ >= 5
    chi = ((obs[keep] - exp_[keep]) ** 2 / exp_[keep]).sum() + \
        (obs[~keep].sum() - exp_[~keep].sum()) ** 2 / max(exp_[~keep].sum(), 1e-9)
    assert stats.chi2.sf(chi, keep.sum()) > 1e-3


def test_indexed_phase_rejects_residues_above_the_index(graph):
    rp, col = graph
    n = len(rp) - 1
    C = oracle.walk_scale(0.5, 1.0 / n, 1.0 / n)
    rmax = oracle.rmax_rule(0.5, 1.0 / n, 1.0 / n, rp[-1])
    off, dest = oracle.walk_index(rp, col, 0.2, C, rmax, seed=1)
    r = np.zeros(n)
    r[3] = 4.0 * rmax * (rp[4] - rp[3])
    with pytest.raises(oracle.OracleError):
        oracle.walk_phase_indexed(n, C, r, off, dest)


def test_zero_hop_index_equals_zero_hop_walk_phase_with_the_same_streams(graph):
    """An index of zero-hop walks (Section 4.1 inside FORA+) served with zero-hop sampling
    equals the simulated zero-hop walk phase exactly under the query's own streams, and is
    about (1 - alpha) the size of the plain index."""
    rp, col = graph
    n = len(rp) - 1
    s = 23
    C = oracle.walk_scale(0.5, 1.0 / n, 1.0 / n)
    rmax = oracle.rmax_rule(0.5, 1.0 / n, 1.0 / n, rp[-1])
    _, residue, _ = oracle.forward_push(rp, col, s, 0.2, rmax)
    off, dest = oracle.walk_index(rp, col, 0.2, C, rmax, seed=5, s_index=s, zero_hop=True)
    cnt_i, acc_i, st_i = oracle.walk_phase_indexed(n, C, residue, off, dest, alpha=0.2,
                                                   zero_hop=True)
    cnt_w, acc_w, st_w = oracle.walk_phase_zero_hop(rp, col, s, 0.2, C, 5, residue)
    np.testing.assert_array_equal(cnt_i, cnt_w)
    np.testing.assert_array_equal(acc_i, acc_w)
    assert st_i.walks == st_w.walks
    off_plain, _ = oracle.walk_index(rp, col, 0.2, C, rmax, seed=5)
    assert 0.75 < off[-1] / off_plain[-1] < 0.85

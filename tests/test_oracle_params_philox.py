"""Pins for the oracle's parameter rules and its Philox generator (CPU only)."""
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("eps,delta,pf", [(0.5, 1 / 2**14, 1 / 2**14), (0.5, 1 / 2**20, 1 / 2**20),
                                          (0.3, 1 / 2**25, 1 / 2**25), (0.1, 1e-3, 1e-2)])
def test_walk_scale_meets_the_chernoff_bound_at_delta(eps, delta, pf):
    """Lemma (layerppr-conc): with omega = r_sum * C the bound of Eq. (relative-error)
    at pi(s,t) = delta is exactly p_f, for any r_sum."""
    C = oracle.walk_scale(eps, delta, pf)
    for rsum in (1.0, 0.37, 1e-3):
        omega = rsum * C
        bound = 2.0 * math.exp(-(eps**2) * omega * delta / (rsum * (2.0 + 2.0 * eps / 3.0)))
        assert bound == pytest.approx(pf, rel=1e-11)


@pytest.mark.parametrize("n,m", [(2**14, 138275), (2**20, 17278754), (2**25, 2**25 * 32)])
def test_rmax_rule_case1_minimises_the_cost_model(n, m):
    """Section 3.2: r_max minimises 1/r_max + m r_max C (push + walk cost) when m r_max <= 1."""
    eps, delta, pf = 0.5, 1.0 / n, 1.0 / n
    C = oracle.walk_scale(eps, delta, pf)
    r = oracle.rmax_rule(eps, delta, pf, m)
    assert m * r <= 1.0
    cost = lambda logr: 1.0 / math.exp(logr) + m * math.exp(logr) * C
    best = minimize_scalar(cost, bracket=(math.log(r) - 3, math.log(r) + 3), tol=1e-12)
    assert math.exp(best.x) == pytest.approx(r, rel=1e-5)


def test_rmax_rule_case2_uses_the_mc_threshold():
    """Case 2 of Section 3.2: when m r_max > 1 the rule falls back to
    eps^2 delta / ((2eps/3+2) log(2/p_f)), i.e. r_max = 1/C (one walk per unit of residue)."""
    eps, delta, pf, m = 1.0, 0.5, 0.5, 100.0
    C = oracle.walk_scale(eps, delta, pf)
    assert m / C > 1.0  # the unconstrained optimum 1/sqrt(mC) has m r > 1
    r = oracle.rmax_rule(eps, delta, pf, m)
    assert r * C == pytest.approx(1.0, rel=1e-14)


def test_rmax_rule_table_values():
    """Values of the rule at the three R-MAT workloads (alpha-independent), as derived by
    hand from Eq. (rmax) with natural log: 2.191e-6, 2.045e-8, 4.062e-10 for
    (n, m) = (2^14, 131072), (2^20, 16777216), (2^25, 1073741824)."""
    for n, m, want in [(2**14, 131072, 2.191e-6), (2**20, 16777216, 2.045e-8),
                       (2**25, 1073741824, 4.062e-10)]:
        assert oracle.rmax_rule(0.5, 1.0 / n, 1.0 / n, m) == pytest.approx(want, rel=2e-3)


@pytest.mark.parametrize("alpha", [0.2, 0.15, 0.5, 1e-9, 0.999999])
def test_alpha_threshold_brackets_alpha(alpha):
    t = oracle.alpha_threshold(alpha)
    assert t / 2**32 <= alpha < (t + 1) / 2**32


def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_philox_outputs_look_uniform():
    """Sanity: over 4096 counters the output bits are balanced (a wrong rotation of words
    or a missing round shows up as strong bias or repeats)."""
    outs = np.array([oracle.philox4x32_10([i, 7, 9, 11], [1, 2]) for i in range(4096)])
    assert len(np.unique(outs[:, 0])) == 4096
    bits = np.unpackbits(outs.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.01

"""What the learned r_max gains over the rule, with the accuracy re-checked (needs a GPU).

Trains the network on the GPU from the method's own measurements (2048 sources of a
2^16-node R-MAT graph at 8 r_max values around the rule) and evaluates it on 512
held-out sources: the modelled cost (per-unit costs calibrated from the measured phase
times) must drop, and the learned queries stay eps-accurate against power iteration.
"""
import numpy as np
import pytest

import inputs
import oracle
from oracle import exact

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1908_10583_gb300 as fora  # noqa: E402
from paper_1908_10583_gb300 import build as fbuild  # noqa: E402
from paper_1908_10583_gb300 import learned_rmax as lr  # noqa: E402


def test_learned_rmax_gains_over_the_rule_and_stays_accurate():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fbuild.build()
    rp, col = inputs.rmat_csr(16, 16, 12)
    n = len(rp) - 1
    g = fora.Graph(rp, col)
    params = fora.Params.make(eps=0.5, k=100, seed=3)
    pool = inputs.uniform_sources(n, 2048 + 512, 4242)
    tr, ev = pool[:2048], pool[2048:]
    cnt, runs, _ = lr.measure(g, tr, params, batch=256)
    coef = lr.calibrate(runs)
    costs = lr.cost(cnt, coef)
    y = lr.labels(costs)
    model, hist = lr.train(g.features(tr, params), y, epochs=60)
    assert hist[-1] < hist[0]
    res = lr.evaluate(g, model, ev, params, coef, batch=256)
    print("learned r_max on held-out sources:", res)
    assert res["cost_gain"] > 0.0
    # accuracy re-checked on held-out sources (Lemma (layerppr-conc) holds for any r_max)
    src = ev[:6]
    truth = exact.power_iteration(rp, col, 0.2, src)
    S = len(src)
    _, _, st = g.ssppr_batch_learned(src, params, model)
    for i in range(S):
        q = oracle.ssppr(rp, col, src[i], rmax=st[i].rmax, k=100, seed=3)
        big = truth[i] >= 1.0 / n
        assert (np.abs(q.est[big] - truth[i][big]) / truth[i][big]).max() <= 0.5

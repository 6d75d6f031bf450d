"""The output-layer anchoring of the learned r_max (host arithmetic, no GPU): with share
lam of the per-source deviations kept, the network's output becomes
log2(c) + lam (y - mean y), y the original output; lam = 0 is the constant c itself.
Checked through the oracle's forward pass with BF16 weights."""
import numpy as np
import pytest

from oracle import learn
from paper_1908_10583_gb300 import learned_rmax as lr


def _network(seed):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(learn.N_PARAMS) * 0.2).astype(np.float32)
    p[learn.OFF_B3] = np.float32(0.37)
    norm = np.concatenate([np.zeros(learn.N_FEATURES), np.ones(learn.N_FEATURES)]).astype(np.float32)
    X = rng.standard_normal((300, learn.N_FEATURES)).astype(np.float32)
    return p, norm, X


def test_output_layer_offsets():
    assert (lr.OFF_W3, lr.OFF_B3) == (learn.OFF_W3, learn.OFF_B3)
    assert lr.OFF_B3 + 1 == learn.N_PARAMS


@pytest.mark.parametrize("lam", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("const_mult", [0.5, 2.0 ** 0.5, 3.0])
def test_anchored_output(lam, const_mult):
    p, norm, X = _network(5)
    y, _ = learn.forward(p, norm, X)
    q = lr.anchored(p, y, const_mult, lam)
    y2, _ = learn.forward(q, norm, X)
    mu = np.clip(y, -3.0, 3.0).mean()
    want = np.log2(const_mult) + lam * (y - mu)
    # only b3 is rounded differently: BF16 of the moved bias against lam * BF16 of the old one
    tol = 2.0 ** -8 * (abs(float(q[learn.OFF_B3])) + lam * abs(float(p[learn.OFF_B3]))) + 1e-9
    assert np.max(np.abs(y2 - want)) <= tol
    # the rest of the network is unchanged; W3 is scaled exactly
    assert np.array_equal(q[:learn.OFF_W3], p[:learn.OFF_W3])
    assert np.array_equal(q[learn.OFF_W3:learn.OFF_B3], p[learn.OFF_W3:learn.OFF_B3] * np.float32(lam))


def test_anchor_zero_is_the_constant():
    p, norm, X = _network(6)
    y, _ = learn.forward(p, norm, X)
    y2, _ = learn.forward(lr.anchored(p, y, 0.5, 0.0), norm, X)
    assert np.all(y2 == -1.0)  # log2(0.5), exact in BF16, whatever the features

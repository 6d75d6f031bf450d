"""Pins for the learned r_max oracle (features, BF16 rounding, MLP gradients), CPU only."""
import math

import numpy as np
import pytest

import inputs
from oracle import learn


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-6, 6, 20000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, -3.1415927],
                                 dtype=np.float32)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(learn.bf16(x), want)


def test_gradient_matches_finite_differences():
    """Without the BF16 rounding the network is smooth away from ReLU kinks: central
    differences in FP64 pin every block of the analytic gradient."""
    rng = np.random.default_rng(1)
    p = (rng.standard_normal(learn.N_PARAMS) * 0.3).astype(np.float64)
    norm = np.concatenate([np.zeros(16), np.ones(16)]).astype(np.float32)
    X = rng.standard_normal((40, 16)).astype(np.float32)
    T = rng.standard_normal(40)
    g, _ = learn.gradient(p, norm, X, T, rounding=False)
    h = 1e-6
    idx = np.concatenate([rng.choice(np.arange(learn.OFF_W1, learn.OFF_B1), 12),
                          rng.choice(np.arange(learn.OFF_B1, learn.OFF_W2), 6),
                          rng.choice(np.arange(learn.OFF_W2, learn.OFF_B2), 12),
                          rng.choice(np.arange(learn.OFF_B2, learn.OFF_W3), 6),
                          rng.choice(np.arange(learn.OFF_W3, learn.OFF_B3), 6), [learn.OFF_B3]])
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (learn.gradient(pp, norm, X, T, rounding=False)[1]
               - learn.gradient(pm, norm, X, T, rounding=False)[1]) / (2 * h)
        assert g[i] == pytest.approx(num, rel=1e-5, abs=1e-9), i


def test_forward_with_rounding_is_close_to_unrounded():
    rng = np.random.default_rng(2)
    p = (rng.standard_normal(learn.N_PARAMS) * 0.2).astype(np.float32)
    norm = np.concatenate([np.zeros(16), np.ones(16)]).astype(np.float32)
    X = rng.standard_normal((100, 16)).astype(np.float32)
    y_r, _ = learn.forward(p, norm, X, rounding=True)
    y_u, _ = learn.forward(p.astype(np.float64), norm, X, rounding=False)
    assert np.abs(y_r - y_u).max() < 0.05 * (np.abs(y_u).max() + 1)


def test_features_by_hand():
    """Star: 0 -> {1, 2, 3}; 1 -> {0}; 2 -> {0, 3}; 3 -> {0}.  alpha = 0.2, r_rule = 0.15:
    d(0) = 3, d_in(0) = 3; neighbours' out-degrees 1 + 2 + 1 = 4, in-degrees 1 + 1 + 2 = 4;
    round-1 residue per edge 0.8/3 = 0.267 exceeds 0.15 d(u) for u = 1, 3 (d = 1) but not
    for u = 2 (0.3): 1-hop frontier of 2 nodes with 1 + 1 out-edges."""
    rp, col = inputs.csr_from_edges(4, [(0, 1), (0, 2), (0, 3), (1, 0), (2, 0), (2, 3), (3, 0)])
    f = learn.features(rp, col, [0], 0.2, 0.15)[0]
    want = [math.log1p(3), math.log1p(3), math.log1p(4), math.log1p(4), math.log1p(2),
            math.log1p(2), math.log(0.15 * 7), math.log(7 / 4)] + [0.0] * 8
    np.testing.assert_allclose(f, np.array(want, dtype=np.float32), rtol=1e-7)

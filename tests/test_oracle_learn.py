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


def hand_network():
    """Parameters and one input of a 16-64-64-1 network worked by hand, where every BF16
    rounding point of the forward pass changes the output if it is dropped or moved.
    Only unit 0 of each layer is used (every other weight and bias is 0), mu = 0,
    sigma = 1, and the input is f0 = 1 + 2^-8 (other features 0).  BF16 keeps 8
    significant bits, so near 1 its values are 1, 1 + 2^-7, ... and 1 + 2^-8 is a tie
    that rounds to even (1.0).  Masters: W1[0][0] = W2[0][0] = W3[0] = 1 + 2^-8 (BF16:
    1.0), b1[0] = b2[0] = 2^-8 + 2^-17 (BF16: 2^-8), b3 = 2^-12 + 2^-25 (BF16: 2^-12).
    With every rounding in place: x0 = 1, z1 = 1 + 2^-8 -> h1 = 1 (tie), z2 = 1 + 2^-8
    -> h2 = 1 (tie), y = 1 + 2^-12 (the output is not rounded)."""
    p = np.zeros(learn.N_PARAMS, dtype=np.float32)
    p[learn.OFF_W1 + 0] = 1 + 2.0 ** -8
    p[learn.OFF_B1 + 0] = 2.0 ** -8 + 2.0 ** -17
    p[learn.OFF_W2 + 0] = 1 + 2.0 ** -8
    p[learn.OFF_B2 + 0] = 2.0 ** -8 + 2.0 ** -17
    p[learn.OFF_W3 + 0] = 1 + 2.0 ** -8
    p[learn.OFF_B3] = 2.0 ** -12 + 2.0 ** -25
    norm = np.concatenate([np.zeros(16), np.ones(16)]).astype(np.float32)
    x = np.zeros((1, 16), dtype=np.float32)
    x[0, 0] = 1 + 2.0 ** -8
    return p, norm, x


def test_forward_rounding_points_by_hand():
    """Each misplaced rounding gives another output: dropping the input rounding makes
    z1 = 1 + 2^-7 (h1 = 1 + 2^-7, y about 1.0078); unrounded W1 or b1 push z1 above the
    tie (h1 = 1 + 2^-7); an unrounded h1 makes z2 = 1 + 2^-7; an unrounded W2 or b2 push
    z2 above its tie; an unrounded h2 gives y = 1 + 2^-8 + 2^-12; unrounded W3 or b3 add
    2^-8 or 2^-25; rounding y itself would give 1.0."""
    p, norm, x = hand_network()
    y, _ = learn.forward(p, norm, x, rounding=True)
    assert y[0] == 1 + 2.0 ** -12
    # without any rounding: the exact FP64 value of the same arithmetic
    e = 1 + 2.0 ** -8
    z1 = e * e + 2.0 ** -8 + 2.0 ** -17
    z2 = e * z1 + 2.0 ** -8 + 2.0 ** -17
    want = e * z2 + 2.0 ** -12 + 2.0 ** -25
    y_u, _ = learn.forward(p.astype(np.float64), norm, x, rounding=False)
    assert y_u[0] == want

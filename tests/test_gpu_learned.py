"""Learned r_max on the GPU against the numpy oracle (needs a GPU)."""
import numpy as np
import pytest

import inputs
import oracle
from oracle import exact, learn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1908_10583_gb300 as fora  # noqa: E402
from paper_1908_10583_gb300 import build as fbuild  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fbuild.build()
    fora.load()


@pytest.fixture(scope="module")
def rmat14():
    rp, col = inputs.rmat_csr(14, 8, 1)
    return rp, col, fora.Graph(rp, col)


def test_features_match_oracle(rmat14):
    rp, col, g = rmat14
    n = len(rp) - 1
    src = np.concatenate([inputs.uniform_sources(n, 60, 4), [int(np.argmax(np.diff(rp)))]])
    p = fora.Params.make()
    got = g.features(src, p)
    want = learn.features(rp, col, src, 0.2, g.resolve(p)[0])
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=0)


def _random_model_and_data(seed, n=300):
    rng = np.random.default_rng(seed)
    m = fora.Model(seed)
    p, _ = m.get()
    norm = np.concatenate([rng.normal(0, 1, 16), rng.uniform(0.5, 2, 16)]).astype(np.float32)
    m.set(p, norm)
    x = rng.normal(0, 2, (n, 16)).astype(np.float32)
    t = rng.normal(0, 1, n).astype(np.float32)
    return m, p, norm, x, t


U32 = 2.0 ** -24  # unit roundoff of FP32


def gamma(k):
    """Bound on the relative error of a k-term FP32 dot product or sum (Higham, Thm. 3.1):
    |fl(sum) - sum| <= gamma_k * sum |terms|, gamma_k = k u / (1 - k u)."""
    return k * U32 / (1 - k * U32)


def unambiguous(z, bound):
    """True where every value within `bound` of z rounds (FP32, then BF16, after ReLU) to
    the same BF16 value and takes the same ReLU branch as z: the device's FP32 sum, which
    lies within the bound, then gives the oracle's activation exactly."""
    lo = learn.bf16(np.maximum(z - bound, 0.0).astype(np.float32))
    hi = learn.bf16(np.maximum(z + bound, 0.0).astype(np.float32))
    return (lo == hi) & ((z - bound > 0) | (z + bound <= 0))


def forward_bounds(p, norm, x):
    """The oracle's forward pass and, per sample, whether the device must reproduce every
    hidden activation exactly, with the bound on |y_device - y_oracle| that follows."""
    y, (xb, z1, h1, z2, h2, (W1, b1, W2, b2, W3, b3)) = learn.forward(p, norm, x)
    m1 = np.abs(xb) @ np.abs(W1).T + np.abs(b1)      # magnitudes of the layer-1 sums
    m2 = np.abs(h1) @ np.abs(W2).T + np.abs(b2)
    my = np.abs(h2) @ np.abs(W3) + abs(b3)
    slack = 1.01  # covers the oracle's own FP64 rounding
    ok = (unambiguous(z1, slack * gamma(17) * m1).all(1) &
          unambiguous(z2, slack * gamma(65) * m2).all(1))
    return y, ok, slack * gamma(65) * my, (xb, z1, h1, z2, h2, (W1, b1, W2, b2, W3, b3))


def test_hand_worked_network_on_the_device():
    """The hand-worked case of the oracle pins (every BF16 rounding point matters) gives
    exactly y = 1 + 2^-12 on the device too."""
    from tests.test_oracle_learn import hand_network
    p, norm, x = hand_network()
    m = fora.Model(0)
    m.set(p, norm)
    assert m.predict(x)[0] == np.float32(1 + 2.0 ** -12)


def test_forward_matches_oracle_per_sample():
    """Per sample, within the FP32 accumulation bound of the output layer, wherever the
    hidden activations are unambiguous (no FP32 sum within its error bound of a BF16
    rounding boundary or of the ReLU kink; 128 hidden units per sample, so about a third
    of random samples qualify, and hundreds are checked)."""
    m, p, norm, x, t = _random_model_and_data(3, n=4000)
    y_gpu = m.predict(x).astype(np.float64)
    y_ref, ok, bound, _ = forward_bounds(p, norm, x)
    assert ok.sum() >= 500, ok.sum()
    err = np.abs(y_gpu - y_ref)[ok]
    assert np.all(err <= bound[ok] + U32 * np.abs(y_ref[ok])), (err / bound[ok]).max()
    # the rest still differ by at most a few BF16 steps of one activation
    assert np.abs(y_gpu - y_ref).max() < 0.05 * (np.abs(y_ref).max() + 1)


def gradient_bound(p, norm, x, t, y_gpu_bound, tiles):
    """Per-entry bound on |grad_device - grad_oracle| for samples whose activations agree:
    the FP32 errors of y, dy, dz2 = dy W3, dz1 = W2^T dz2 and of each sum over samples,
    propagated by first-order error analysis (bounds of products add |a| E(b) + |b| E(a))."""
    y, (xb, z1, h1, z2, h2, (W1, b1, W2, b2, W3, b3)) = learn.forward(p, norm, x)
    S = len(t)
    err = y - t
    e_err = y_gpu_bound + 2 * U32 * np.abs(err)
    dy = err / S
    e_dy = (e_err + 3 * U32 * np.abs(err)) / S
    act2 = (z2 > 0).astype(np.float64)
    act1 = (z1 > 0).astype(np.float64)
    dz2 = np.outer(dy, W3) * act2
    e_dz2 = np.outer(e_dy, np.abs(W3)) * act2 + U32 * np.abs(dz2)
    dz1 = (dz2 @ W2) * act1
    e_dz1 = ((e_dz2 @ np.abs(W2)) + gamma(64) * (np.abs(dz2) @ np.abs(W2))) * act1
    gs = gamma(64 + tiles)  # each term passes through <= 64 in-tile and `tiles` tile additions
    g = np.zeros(learn.N_PARAMS)
    g[learn.OFF_W3:learn.OFF_B3] = e_dy @ np.abs(h2) + gs * (np.abs(dy) @ np.abs(h2))
    g[learn.OFF_B3] = e_dy.sum() + gs * np.abs(dy).sum()
    g[learn.OFF_W2:learn.OFF_B2] = (e_dz2.T @ np.abs(h1) + gs * (np.abs(dz2).T @ np.abs(h1))).ravel()
    g[learn.OFF_B2:learn.OFF_W3] = e_dz2.sum(0) + gs * np.abs(dz2).sum(0)
    g[learn.OFF_W1:learn.OFF_B1] = (e_dz1.T @ np.abs(xb) + gs * (np.abs(dz1).T @ np.abs(xb))).ravel()
    g[learn.OFF_B1:learn.OFF_W2] = e_dz1.sum(0) + gs * np.abs(dz1).sum(0)
    return g


def test_gradient_matches_oracle_element_by_element():
    """Every one of the 5313 gradient entries within its own FP32-vs-FP64 error bound (a
    wrong sign, a transposed block or a dropped term moves an entry by about its own
    size, far outside the bound), on samples whose hidden activations are unambiguous."""
    m, p, norm, x, t = _random_model_and_data(5, n=3000)
    _, ok, ybound, _ = forward_bounds(p, norm, x)
    x, t = x[ok], t[ok]
    assert len(t) >= 300
    S = len(t)
    g_gpu, loss_gpu = m.gradient(x, t)
    g_ref, loss_ref = learn.gradient(p, norm, x, t)
    _, _, ybound, _ = forward_bounds(p, norm, x)
    ybound = ybound + U32 * np.abs(learn.forward(p, norm, x)[0])
    tiles = (S + fora_tile() - 1) // fora_tile()
    bound = gradient_bound(p, norm, x, t, ybound, tiles) * 1.05 + 1e-30
    diff = np.abs(g_gpu.astype(np.float64) - g_ref)
    worst = int(np.argmax(diff / bound))
    assert np.all(diff <= bound), (worst, g_gpu[worst], g_ref[worst], bound[worst])
    # the bound is sharp: far below the entries themselves where they are not tiny
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    assert np.median(bound[big] / np.abs(g_ref[big])) < 1e-2
    assert loss_gpu == pytest.approx(loss_ref, rel=1e-5)


def fora_tile():
    return 64  # samples per block of the backward kernel (one partial gradient per tile)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(7)
    x = rng.normal(0, 1, (4096, 16)).astype(np.float32)
    t = (np.tanh(x[:, 0]) + 0.5 * x[:, 1] - 0.25 * x[:, 2] * x[:, 3]).astype(np.float32)
    m = fora.Model(11)
    hist = m.train(x, t, epochs=60, batch=256, lr=3e-3, seed=1)
    assert hist[-1] < 0.1 * hist[0]
    assert hist[-1] < 0.02


def test_learned_query_uses_the_predicted_rmax_and_stays_eps_accurate(rmat14):
    rp, col, g = rmat14
    n = len(rp) - 1
    src = inputs.uniform_sources(n, 8, 808)
    p = fora.Params.make(k=50)
    m = fora.Model(21)
    params, _ = m.get()
    params[learn.OFF_B3] = 0.8  # push r_max up by ~2^0.8 on average
    m.set(params)
    ids, vals, st = g.ssppr_batch_learned(src, p, m)
    r_rule = g.resolve(p)[0]
    pred = np.clip(m.predict(g.features(src, p)), -3, 3)
    np.testing.assert_allclose([s.rmax for s in st], r_rule * np.exp2(pred.astype(np.float64)),
                               rtol=1e-6)
    truth = exact.power_iteration(rp, col, 0.2, src)
    S = len(src)
    dbg = {"reserve": torch.zeros((S, n), dtype=torch.float64, device="cuda"),
           "residue": torch.zeros((S, n), dtype=torch.float64, device="cuda"),
           "estimate": torch.zeros((S, n), dtype=torch.float64, device="cuda")}
    # the same r_max through the per-source entry point: eps-accurate (Lemma (layerppr-conc))
    _, _, st2 = g.ssppr_batch_rmax(src, [s.rmax for s in st], p)
    for i in range(S):
        assert st2[i].rmax == st[i].rmax and st2[i].walks == st[i].walks
    ids3, vals3, _ = g.ssppr_batch_debug(src, p, dbg)
    est_rule = dbg["estimate"].cpu().numpy()
    for i in range(S):
        big = truth[i] >= 1.0 / n
        q = oracle.ssppr(rp, col, src[i], rmax=st[i].rmax, k=50)
        rel = np.abs(q.est[big] - truth[i][big]) / truth[i][big]
        assert rel.max() <= 0.5
        np.testing.assert_allclose(vals[i], q.vals, rtol=0, atol=1e-12)

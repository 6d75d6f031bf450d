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


def test_forward_matches_oracle():
    m, p, norm, x, t = _random_model_and_data(3)
    y_gpu = m.predict(x)
    y_ref, _ = learn.forward(p, norm, x)
    # FP32 vs FP64 accumulation between the same BF16 rounding points
    np.testing.assert_allclose(y_gpu, y_ref, rtol=2e-2, atol=2e-2)
    assert np.abs(y_gpu - y_ref).mean() < 2e-3 * (np.abs(y_ref).mean() + 1)


def test_gradient_matches_oracle():
    m, p, norm, x, t = _random_model_and_data(5)
    g_gpu, loss_gpu = m.gradient(x, t)
    g_ref, loss_ref = learn.gradient(p, norm, x, t)
    assert loss_gpu == pytest.approx(loss_ref, rel=2e-3)
    for lo, hi in [(learn.OFF_W1, learn.OFF_B1), (learn.OFF_B1, learn.OFF_W2),
                   (learn.OFF_W2, learn.OFF_B2), (learn.OFF_B2, learn.OFF_W3),
                   (learn.OFF_W3, learn.OFF_B3), (learn.OFF_B3, learn.N_PARAMS)]:
        a, b = g_gpu[lo:hi].astype(np.float64), g_ref[lo:hi]
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-7, (lo, hi)


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

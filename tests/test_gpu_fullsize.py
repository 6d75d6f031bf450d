"""Parity at full size, in the launch configuration the benchmark times (needs a GPU).

The 2^20-node graph with 256 sources per launch and top-500: sampled sources are
checked against the oracle (push within 1e-12; walk counts, weights, estimates and
top-k bit-exact on the oracle's residues).  The 2^25-node, 1.07e9-edge graph: one
source's push against the oracle, and the walk phase on a sample of the oracle's
residual nodes (the oracle walks only those), bit-exact.
"""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1908_10583_gb300 as fora  # noqa: E402
from paper_1908_10583_gb300 import build as fbuild  # noqa: E402

ATOL_PUSH = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fbuild.build()


def _debug_run(g, sources, p, given=None):
    S, n = len(sources), g.n
    d = {k: torch.zeros((S, n), dtype=dt, device="cuda")
         for k, dt in [("reserve", torch.float64), ("residue", torch.float64),
                       ("count", torch.int32), ("acc", torch.int64), ("estimate", torch.float64)]}
    if given is not None:
        d["reserve"].copy_(given[0])
        d["residue"].copy_(given[1])
    ids, vals, st = g.ssppr_batch_debug(sources, p, d, given_push=given is not None)
    torch.cuda.synchronize()
    return ids, vals, st, d


def test_rmat20_batch256_sampled_sources_match_oracle():
    w = inputs.WORKLOADS["rmat20_deg16"]
    rp, col = inputs.rmat_csr(w["scale"], w["avg_deg"], w["graph_seed"])
    n = len(rp) - 1
    g = fora.Graph(rp, col)
    sources = inputs.uniform_sources(n, w["n_sources"], inputs.SOURCE_SEED)
    p = fora.Params.make(k=w["k"], seed=inputs.WALK_SEED)
    ids, vals, st, d = _debug_run(g, sources, p)
    sample = [0, 97, 255]
    qs = {i: oracle.ssppr(rp, col, sources[i], k=w["k"], seed=inputs.WALK_SEED) for i in sample}
    for i, q in qs.items():
        np.testing.assert_allclose(d["reserve"][i].cpu().numpy(), q.reserve, rtol=0, atol=ATOL_PUSH)
        np.testing.assert_allclose(d["residue"][i].cpu().numpy(), q.residue, rtol=0, atol=ATOL_PUSH)
        assert st[i].pushes == q.push.pushes and st[i].push_rounds == q.push.rounds
    # the same launch with the oracle's reserve and residue in the sampled rows
    res, r = d["reserve"].clone(), d["residue"].clone()
    for i, q in qs.items():
        res[i].copy_(torch.from_numpy(q.reserve))
        r[i].copy_(torch.from_numpy(q.residue))
    ids2, vals2, st2, d2 = _debug_run(g, sources, p, given=(res, r))
    for i, q in qs.items():
        np.testing.assert_array_equal(d2["count"][i].cpu().numpy().view(np.uint32), q.count)
        np.testing.assert_array_equal(d2["acc"][i].cpu().numpy().view(np.uint64), q.acc)
        np.testing.assert_array_equal(d2["estimate"][i].cpu().numpy(), q.est)
        np.testing.assert_array_equal(ids2[i], q.ids)
        np.testing.assert_array_equal(vals2[i], q.vals)
    del d, d2, res, r
    g.close()
    torch.cuda.empty_cache()


def test_rmat25_push_and_sampled_walks_match_oracle():
    w = inputs.WORKLOADS["rmat25_deg32"]
    rp, col = inputs.rmat_csr(w["scale"], w["avg_deg"], w["graph_seed"])
    n = len(rp) - 1
    assert rp[-1] > 1_000_000_000
    g = fora.Graph(rp, col)
    s = int(inputs.uniform_sources(n, 1, inputs.SOURCE_SEED)[0])
    p = fora.Params.make(k=w["k"], seed=inputs.WALK_SEED)
    rmax = g.resolve(p)[0]
    res_o, r_o, pst = oracle.forward_push(rp, col, s, 0.2, rmax)
    ids, vals, st, d = _debug_run(g, [s], p)
    np.testing.assert_allclose(d["reserve"][0].cpu().numpy(), res_o, rtol=0, atol=ATOL_PUSH)
    np.testing.assert_allclose(d["residue"][0].cpu().numpy(), r_o, rtol=0, atol=ATOL_PUSH)
    assert st[0].pushes == pst.pushes and st[0].push_rounds == pst.rounds
    # walks from a sample of the oracle's residual nodes (the 3000 largest residues)
    keep = np.argsort(r_o)[-3000:]
    r_s = np.zeros(n)
    r_s[keep] = r_o[keep]
    C = oracle.walk_scale(0.5, 1.0 / n, 1.0 / n)
    cnt_o, acc_o, wst = oracle.walk_phase(rp, col, s, 0.2, C, inputs.WALK_SEED, r_s)
    ids2, vals2, st2, d2 = _debug_run(g, [s], p, given=(torch.from_numpy(res_o)[None],
                                                      torch.from_numpy(r_s)[None]))
    np.testing.assert_array_equal(d2["count"][0].cpu().numpy().view(np.uint32), cnt_o)
    np.testing.assert_array_equal(d2["acc"][0].cpu().numpy().view(np.uint64), acc_o)
    assert st2[0].walks == wst.walks and st2[0].walk_steps == wst.walk_steps
    est_o = oracle.estimate(res_o, acc_o)
    ids_o, vals_o = oracle.topk(est_o, w["k"])
    np.testing.assert_array_equal(ids2[0], ids_o)
    np.testing.assert_array_equal(vals2[0], vals_o)
    del d, d2
    g.close()
    torch.cuda.empty_cache()

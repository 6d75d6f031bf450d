"""FORA+ walk index (Section 3.3) on the device against the oracle (needs a GPU).

The device index (omega_max(v) stored walk ends per node) equals the oracle's bit for
bit; a query served from it equals the oracle's indexed walk phase bit for bit on the
oracle's residues (counts, fixed-point weights, estimates, top-k); indexed queries stay
eps-accurate against power iteration; an index of zero-hop walks (Section 4.1) serves
zero-hop queries bit-exactly too; and the refusals (a query of the other walk kind, an
r_max above the index's, other parameters, no index) are errors.
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

SEED = 77


@pytest.fixture(scope="module")
def indexed():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fbuild.build()
    rp, col = inputs.rmat_csr(14, 8, 1)
    g = fora.Graph(rp, col)
    p = fora.Params.make(k=50, seed=SEED)
    g.build_index(p)
    yield rp, col, g
    g.close()


def _debug(g, sources, params, given=None):
    S, n = len(sources), g.n
    d = {k: torch.zeros((S, n), dtype=dt, device="cuda")
         for k, dt in [("reserve", torch.float64), ("residue", torch.float64),
                       ("count", torch.int32), ("acc", torch.int64), ("estimate", torch.float64)]}
    if given is not None:
        d["reserve"].copy_(torch.from_numpy(np.ascontiguousarray(given[0])))
        d["residue"].copy_(torch.from_numpy(np.ascontiguousarray(given[1])))
    ids, vals, st = g.ssppr_batch_debug(sources, params, d, given_push=given is not None)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in d.items()}
    out["count"] = out["count"].view(np.uint32)
    out["acc"] = out["acc"].view(np.uint64)
    return ids, vals, st, out


def test_device_index_equals_oracle_index(indexed):
    rp, col, g = indexed
    n = len(rp) - 1
    rmax, C, entries = g.index_info()
    assert rmax == oracle.rmax_rule(0.5, 1.0 / n, 1.0 / n, rp[-1])
    assert C == oracle.walk_scale(0.5, 1.0 / n, 1.0 / n)
    off, dest = g.index_export()
    off_o, dest_o = oracle.walk_index(rp, col, 0.2, C, rmax, SEED)
    assert entries == off_o[-1] == len(dest)
    np.testing.assert_array_equal(off, off_o)
    np.testing.assert_array_equal(dest.astype(np.int32), dest_o)


def test_indexed_query_bit_exact_on_oracle_residues(indexed):
    rp, col, g = indexed
    n = len(rp) - 1
    rmax, C, _ = g.index_info()
    off_o, dest_o = oracle.walk_index(rp, col, 0.2, C, rmax, SEED)
    sources = inputs.uniform_sources(n, 6, 8080)
    res = np.zeros((len(sources), n))
    r = np.zeros((len(sources), n))
    for i, s in enumerate(sources):
        res[i], r[i], _ = oracle.forward_push(rp, col, int(s), 0.2, rmax)
    p = fora.Params.make(k=50, seed=1, flags=fora.FORA_USE_INDEX)
    ids, vals, st, out = _debug(g, sources, p, given=(res, r))
    for i in range(len(sources)):
        cnt_o, acc_o, wst = oracle.walk_phase_indexed(n, C, r[i], off_o, dest_o)
        np.testing.assert_array_equal(out["count"][i], cnt_o)
        np.testing.assert_array_equal(out["acc"][i], acc_o)
        est_o = oracle.estimate(res[i], acc_o)
        np.testing.assert_array_equal(out["estimate"][i], est_o)
        ids_o, vals_o = oracle.topk(est_o, 50)
        np.testing.assert_array_equal(ids[i], ids_o)
        np.testing.assert_array_equal(vals[i], vals_o)
        assert st[i].walks == wst.walks and st[i].walk_steps == 0


def test_indexed_queries_are_eps_accurate(indexed):
    """Def. 1 for every t with pi >= delta, the pushes run by the device, walks from the
    index (Section 3.3: the index does not change the guarantee of Lemma (layerppr-conc)),
    also through a pipelined batch."""
    rp, col, g = indexed
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 8, 9090)
    truth = exact.power_iteration(rp, col, 0.2, sources)
    p = fora.Params.make(k=50, flags=fora.FORA_USE_INDEX)
    _, _, st, out = _debug(g, sources, p)
    for i in range(len(sources)):
        big = truth[i] >= 1.0 / n
        rel = np.abs(out["estimate"][i][big] - truth[i][big]) / truth[i][big]
        assert rel.max() <= 0.5
        assert st[i].walks > 0 and st[i].walk_steps == 0
    many = inputs.uniform_sources(n, 96, 9191)
    ids1, vals1, _ = g.ssppr_batch(many, p)
    try:
        g.tune("pipeline", 2)
        ids2, vals2, _ = g.ssppr_batch(many, p)
    finally:
        g.tune("pipeline", 1)
    np.testing.assert_allclose(vals2, vals1, rtol=0, atol=2e-12)


def test_index_refusals(indexed):
    rp, col, g = indexed
    n = len(rp) - 1
    rmax, _, _ = g.index_info()
    src = inputs.uniform_sources(n, 2, 7)
    with pytest.raises(fora.FORAError):  # a plain index serves no zero-hop query
        g.ssppr_batch(src, fora.Params.make(k=10, flags=fora.FORA_USE_INDEX | fora.FORA_ZERO_HOP))
    with pytest.raises(fora.FORAError):  # a larger r_max needs more walks than stored
        g.ssppr_batch(src, fora.Params.make(k=10, rmax=2 * rmax, flags=fora.FORA_USE_INDEX))
    with pytest.raises(fora.FORAError):  # other eps: other C
        g.ssppr_batch(src, fora.Params.make(k=10, eps=0.3, flags=fora.FORA_USE_INDEX))
    g2 = fora.Graph(rp, col)
    try:
        with pytest.raises(fora.FORAError):  # no index
            g2.ssppr_batch(src, fora.Params.make(k=10, flags=fora.FORA_USE_INDEX))
        assert g2.index_info() == (0.0, 0.0, 0)
    finally:
        g2.close()


def test_zero_hop_index_bit_exact(indexed):
    """An index of zero-hop walks (FORA_ZERO_HOP at build, Section 4.1) equals the oracle's,
    and a zero-hop query served from it equals the oracle's zero-hop indexed phase bit for
    bit on the oracle's residues; a plain query is refused by it."""
    rp, col, g = indexed
    n = len(rp) - 1
    try:
        g.build_index(fora.Params.make(k=50, seed=SEED, flags=fora.FORA_ZERO_HOP))
        rmax, C, entries = g.index_info()
        off, dest = g.index_export()
        off_o, dest_o = oracle.walk_index(rp, col, 0.2, C, rmax, SEED, zero_hop=True)
        np.testing.assert_array_equal(off, off_o)
        np.testing.assert_array_equal(dest.astype(np.int32), dest_o)
        sources = inputs.uniform_sources(n, 4, 7070)
        res = np.zeros((len(sources), n))
        r = np.zeros((len(sources), n))
        for i, s in enumerate(sources):
            res[i], r[i], _ = oracle.forward_push(rp, col, int(s), 0.2, rmax)
        p = fora.Params.make(k=50, seed=1, flags=fora.FORA_USE_INDEX | fora.FORA_ZERO_HOP)
        ids, vals, st, out = _debug(g, sources, p, given=(res, r))
        for i in range(len(sources)):
            cnt_o, acc_o, _ = oracle.walk_phase_indexed(n, C, r[i], off_o, dest_o, alpha=0.2,
                                                        zero_hop=True)
            np.testing.assert_array_equal(out["count"][i], cnt_o)
            np.testing.assert_array_equal(out["acc"][i], acc_o)
            est_o = oracle.estimate_zero_hop(res[i], r[i], acc_o, 0.2)
            np.testing.assert_array_equal(out["estimate"][i], est_o)
            ids_o, vals_o = oracle.topk(est_o, 50)
            np.testing.assert_array_equal(ids[i], ids_o)
            np.testing.assert_array_equal(vals[i], vals_o)
        with pytest.raises(fora.FORAError):
            g.ssppr_batch(sources, fora.Params.make(k=10, flags=fora.FORA_USE_INDEX))
    finally:
        g.build_index(fora.Params.make(k=50, seed=SEED))

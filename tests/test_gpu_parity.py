"""CUDA path vs the CPU oracle, element by element, through the C ABI (needs a GPU).

Tolerances: reserves and residues of the push within 1e-12 absolute (FP64 atomics
reorder the sums); walk counts, fixed-point walk weights, estimates and top-k
bit-exact when both sides run the walk phase on the oracle's reserve and residue.
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

ATOL_PUSH = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fbuild.build()
    fora.load()


def cuda_zeros(shape, dtype):
    return torch.zeros(shape, dtype=dtype, device="cuda")


def run_debug(g, sources, params, given=None):
    """Batched query with all intermediate arrays; given = (reserve, residue) numpy [S, n]."""
    S, n = len(sources), g.n
    dbg = dict(reserve=cuda_zeros((S, n), torch.float64), residue=cuda_zeros((S, n), torch.float64),
               count=cuda_zeros((S, n), torch.int32), acc=cuda_zeros((S, n), torch.int64),
               estimate=cuda_zeros((S, n), torch.float64))
    if given is not None:
        dbg["reserve"].copy_(torch.from_numpy(np.ascontiguousarray(given[0])))
        dbg["residue"].copy_(torch.from_numpy(np.ascontiguousarray(given[1])))
    ids, vals, st = g.ssppr_batch_debug(sources, params, dbg, given_push=given is not None)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in dbg.items()}
    out["count"] = out["count"].view(np.uint32)
    out["acc"] = out["acc"].view(np.uint64)
    return ids, vals, st, out


@pytest.fixture(scope="module")
def rmat14():
    rp, col = inputs.rmat_csr(14, 8, 1)
    return rp, col, fora.Graph(rp, col)


def test_device_philox_matches_oracle_and_published_vectors():
    rng = np.random.default_rng(0)
    rows = rng.integers(0, 2**32, size=(500, 6), dtype=np.uint64).astype(np.uint32)
    kat = np.array([[0, 0, 0, 0, 0, 0], [0xffffffff] * 6,
                    [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344, 0xa4093822, 0x299f31d0]],
                   dtype=np.uint32)
    rows = np.vstack([kat, rows])
    dev = fora.philox(rows)
    for r, d in zip(rows, dev):
        np.testing.assert_array_equal(d, oracle.philox4x32_10(r[:4], r[4:]))
    np.testing.assert_array_equal(dev[0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8])


def test_resolved_parameters_are_bit_identical_to_the_oracle(rmat14):
    rp, col, g = rmat14
    n = len(rp) - 1
    for eps in (0.5, 0.3, 0.1):
        p = fora.Params.make(eps=eps)
        rmax, C, t = g.resolve(p)
        assert rmax == oracle.rmax_rule(eps, 1.0 / n, 1.0 / n, rp[-1])
        assert C == oracle.walk_scale(eps, 1.0 / n, 1.0 / n)
        assert t == oracle.alpha_threshold(0.2)


def hot_count(col, n):
    """Hot nodes of the push (the up to 128 of highest in-degree, each >= 64, ties at the
    cut left out), counted from the in-degrees."""
    indeg = np.bincount(np.asarray(col, dtype=np.int64), minlength=n)
    cut = 64
    if n > 128:
        cut = max(cut, int(np.sort(indeg)[n - 129]) + 1)
    return int((indeg >= cut).sum())


@pytest.mark.parametrize("spread_hot", [1, 0])
def test_push_matches_oracle(rmat14, spread_hot):
    """Push reserves and residues against the oracle, with the hot-node sums of the
    spread (1, the default) and with one atomic per push (0)."""
    rp, col, g = rmat14
    n = len(rp) - 1
    nhot = g.tuning("hot_nodes")
    assert nhot == hot_count(col, n) and 0 < nhot <= 128
    sources = inputs.uniform_sources(n, 10, inputs.SOURCE_SEED)
    p = fora.Params.make(k=50)
    g.tune("spread_hot", spread_hot)
    try:
        ids, vals, st, out = run_debug(g, sources, p)
    finally:
        g.tune("spread_hot", 1)
    rmax = g.resolve(p)[0]
    for i, s in enumerate(sources):
        res, r, pst = oracle.forward_push(rp, col, s, 0.2, rmax)
        np.testing.assert_allclose(out["reserve"][i], res, rtol=0, atol=ATOL_PUSH)
        np.testing.assert_allclose(out["residue"][i], r, rtol=0, atol=ATOL_PUSH)
        # the same nodes were pushed: the frontiers agreed round by round
        assert st[i].pushes == pst.pushes and st[i].edge_pushes == pst.edge_pushes
        assert st[i].push_rounds == pst.rounds
        assert st[i].rsum == pytest.approx(pst.rsum, abs=1e-12)


@pytest.mark.parametrize("walk_blocks", [3, 4, 5])
def test_walks_and_topk_bit_exact_on_oracle_residues(rmat14, walk_blocks):
    """Every walk kernel instance (3, 4 or 5 resident blocks per SM) consumes each walk's
    Philox words exactly as the oracle's word-by-word walk does."""
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 10, inputs.SOURCE_SEED)
    p = fora.Params.make(k=50, seed=inputs.WALK_SEED)
    qs = [oracle.ssppr(rp, col, s, k=50, seed=inputs.WALK_SEED) for s in sources]
    given = (np.stack([q.reserve for q in qs]), np.stack([q.residue for q in qs]))
    g.tune("walk_blocks", walk_blocks)
    try:
        ids, vals, st, out = run_debug(g, sources, p, given=given)
    finally:
        g.tune("walk_blocks", 4)
    for i, q in enumerate(qs):
        np.testing.assert_array_equal(out["count"][i], q.count)
        np.testing.assert_array_equal(out["acc"][i], q.acc)
        np.testing.assert_array_equal(out["estimate"][i], q.est)
        np.testing.assert_array_equal(ids[i], q.ids)
        np.testing.assert_array_equal(vals[i], q.vals)
        assert st[i].walks == q.walk.walks
        assert st[i].walk_steps == q.walk.walk_steps
        assert st[i].residual_nodes == q.walk.residual_nodes


def test_full_query_matches_oracle(rmat14):
    """Without injected residues: same counts (omega_v = ceil(r C) is insensitive to
    the last bits of r), estimates within the push tolerance, same top-k up to near-ties."""
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 10, inputs.SOURCE_SEED)
    p = fora.Params.make(k=50, seed=inputs.WALK_SEED)
    ids, vals, st, out = run_debug(g, sources, p)
    for i, s in enumerate(sources):
        q = oracle.ssppr(rp, col, s, k=50, seed=inputs.WALK_SEED)
        np.testing.assert_array_equal(out["count"][i], q.count)
        np.testing.assert_allclose(out["estimate"][i], q.est, rtol=0, atol=ATOL_PUSH)
        np.testing.assert_allclose(vals[i], q.est[ids[i]], rtol=0, atol=ATOL_PUSH)
        kth = q.vals[-1]
        sure = set(np.flatnonzero(q.est > kth + 2 * ATOL_PUSH).tolist())
        assert sure <= set(ids[i].tolist())
        assert np.all(q.est[ids[i]] >= kth - 2 * ATOL_PUSH)


def test_single_and_batch_agree(rmat14):
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 6, 7)
    p = fora.Params.make(k=50, seed=11)
    ids_b, vals_b, st_b, out_b = run_debug(g, sources, p)
    given = (out_b["reserve"], out_b["residue"])
    # the same residues, one source at a time: bit-exact walk phase and top-k
    for i, s in enumerate(sources):
        ids1, vals1, _, out1 = run_debug(g, [s], p, given=(given[0][i:i + 1], given[1][i:i + 1]))
        np.testing.assert_array_equal(out1["count"][0], out_b["count"][i])
        np.testing.assert_array_equal(out1["acc"][0], out_b["acc"][i])
        np.testing.assert_array_equal(ids1[0], ids_b[i])
        # and the public single-source entry point agrees up to the push rounding
        ids2, vals2, st2 = g.ssppr(s, p)
        np.testing.assert_allclose(vals2, vals_b[i], rtol=0, atol=ATOL_PUSH)
        assert st2.walks == st_b[i].walks


def test_eps_accuracy_against_power_iteration(rmat14):
    """Def. 1 / Lemma (layerppr-conc): relative error <= eps for every t with pi >= delta."""
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 10, inputs.SOURCE_SEED)
    truth = exact.power_iteration(rp, col, 0.2, sources)
    p = fora.Params.make(k=50, eps=0.5)
    _, _, _, out = run_debug(g, sources, p)
    fails = 0
    for i in range(len(sources)):
        big = truth[i] >= 1.0 / n
        rel = np.abs(out["estimate"][i][big] - truth[i][big]) / truth[i][big]
        fails += int(rel.max() > 0.5)
    assert fails == 0


def test_hub_source_and_mc_mode(rmat14):
    """The largest-degree node as source (chunked hub pushes) and r_max = 1 (no push,
    pure Monte-Carlo), both against the oracle on the same residues."""
    rp, col, g = rmat14
    deg = np.diff(rp)
    hub = int(np.argmax(deg))
    assert deg[hub] > 256
    for rmax in (0.0, 1.0):
        p = fora.Params.make(k=20, rmax=rmax, seed=3)
        q = oracle.ssppr(rp, col, hub, k=20, rmax=rmax, seed=3)
        ids, vals, st, out = run_debug(g, [hub], p)
        np.testing.assert_allclose(out["reserve"][0], q.reserve, rtol=0, atol=ATOL_PUSH)
        np.testing.assert_array_equal(out["count"][0], q.count)
        np.testing.assert_array_equal(ids[0], q.ids)
        assert st[0].push_rounds == q.push.rounds


def test_tiny_graphs_and_ragged_sizes():
    # hand-worked triangle (round-synchronous push), see the oracle pins
    rp, col = inputs.csr_from_edges(3, [(0, 1), (0, 2), (1, 2), (2, 0)])
    g = fora.Graph(rp, col)
    p = fora.Params.make(alpha=0.5, rmax=0.1, k=3, delta=0.5, pf=0.5)
    ids, vals, st, out = run_debug(g, [0], p)
    np.testing.assert_array_equal(out["reserve"][0], [0.5, 0.125, 0.1875])
    np.testing.assert_array_equal(out["residue"][0], [0.1875, 0.0, 0.0])
    assert st[0].push_rounds == 3
    q = oracle.ssppr(rp, col, 0, alpha=0.5, rmax=0.1, k=3, delta=0.5, pf=0.5)
    np.testing.assert_array_equal(out["count"][0], q.count)
    np.testing.assert_array_equal(ids[0], q.ids)
    # one node with a self-loop; k = n
    g1 = fora.Graph(np.array([0, 1]), np.array([0], dtype=np.int32))
    ids, vals, _ = g1.ssppr(0, fora.Params.make(k=1, delta=0.5, pf=0.5))
    assert ids[0] == 0 and vals[0] == pytest.approx(1.0, abs=1e-12)
    # a ragged random graph (n not a power of two), k = n, several sources
    rng = np.random.default_rng(5)
    n = 1013
    edges = [(v, int(u)) for v in range(n) for u in rng.integers(0, n, size=1 + rng.poisson(3))]
    rp, col = inputs.csr_from_edges(n, edges)
    g2 = fora.Graph(rp, col)
    src = [0, 1012, 500]
    p = fora.Params.make(k=n, seed=9)
    ids, vals, st, out = run_debug(g2, src, p)
    for i, s in enumerate(src):
        q = oracle.ssppr(rp, col, s, k=n, seed=9)
        np.testing.assert_allclose(out["reserve"][i], q.reserve, rtol=0, atol=ATOL_PUSH)
        np.testing.assert_array_equal(out["count"][i], q.count)
        assert sorted(ids[i].tolist()) == list(range(n))


@pytest.mark.parametrize("n,nrows,k", [(1, 1, 1), (1000, 3, 1000), (5000, 4, 500),
                                       (300_000, 2, 4096), (2**20, 1, 500)])
def test_standalone_topk_bit_exact(n, nrows, k):
    rng = np.random.default_rng(n)
    est = rng.integers(0, 50, size=(nrows, n)) / 64.0  # heavy ties
    est[:, :: 7] = rng.random((nrows, len(range(0, n, 7))))
    ids, vals = fora.topk(torch.from_numpy(est).cuda(), k)
    ids, vals = ids.cpu().numpy(), vals.cpu().numpy()
    for r in range(nrows):
        order = np.lexsort((np.arange(n), -est[r]))[:k]
        np.testing.assert_array_equal(ids[r], order)
        np.testing.assert_array_equal(vals[r], est[r][order])


def test_errors_are_reported(rmat14):
    rp, col, g = rmat14
    with pytest.raises(fora.FORAError) as e:
        g.ssppr(len(rp), fora.Params.make())
    assert e.value.code == fora.FORA_ERR_BAD_ARG
    with pytest.raises(fora.FORAError):
        g.ssppr(0, fora.Params.make(alpha=1.0))
    with pytest.raises(fora.FORAError):
        g.ssppr(0, fora.Params.make(k=5000))
    # the graph stays usable after a rejected call
    ids, vals, st = g.ssppr(0, fora.Params.make(k=5))
    assert len(ids) == 5


def test_zero_hop_bit_exact_on_oracle_residues(rmat14):
    """Walk phase with zero-hop pruning (Section 4.1) on the oracle's residues."""
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 6, 55)
    p = fora.Params.make(k=50, seed=17, flags=fora.FORA_ZERO_HOP)
    qs = [oracle.ssppr(rp, col, s, k=50, seed=17, zero_hop=True) for s in sources]
    given = (np.stack([q.reserve for q in qs]), np.stack([q.residue for q in qs]))
    ids, vals, st, out = run_debug(g, sources, p, given=given)
    for i, q in enumerate(qs):
        np.testing.assert_array_equal(out["count"][i], q.count)
        np.testing.assert_array_equal(out["acc"][i], q.acc)
        np.testing.assert_array_equal(out["estimate"][i], q.est)
        np.testing.assert_array_equal(ids[i], q.ids)
        assert st[i].walks == q.walk.walks and st[i].walk_steps == q.walk.walk_steps
    # full query: eps-accurate against power iteration, and fewer walks than plain FORA
    truth = exact.power_iteration(rp, col, 0.2, sources)
    _, _, st_p, _ = run_debug(g, sources, fora.Params.make(k=50, seed=17))
    _, _, st_z, out_z = run_debug(g, sources, p)
    for i in range(len(sources)):
        big = truth[i] >= 1.0 / n
        rel = np.abs(out_z["estimate"][i][big] - truth[i][big]) / truth[i][big]
        assert rel.max() <= 0.5
        assert st_z[i].walks < 0.85 * st_p[i].walks


def test_topk_fora_matches_oracle(rmat14):
    """Top-k FORA (Alg. 5): the same stopping round and delta per source, the same
    top-k up to near-ties, and Def. 2 against power iteration."""
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 6, 909)
    truth = exact.power_iteration(rp, col, 0.2, sources)
    for k in (20, 100):
        p = fora.Params.make(k=k, seed=5)
        ids, vals, st, iters = g.topk_fora(sources, p)
        for i, s in enumerate(sources):
            q = oracle.topk_fora(rp, col, s, k, seed=5)
            assert iters[i] == q.iterations
            np.testing.assert_allclose(vals[i], q.vals, rtol=0, atol=ATOL_PUSH)
            kth = q.vals[-1]
            sure = set(np.flatnonzero(q.est > kth + 2 * ATOL_PUSH).tolist())
            assert sure <= set(ids[i].tolist())
            true_sorted = np.sort(truth[i])[::-1]
            for j, v in enumerate(ids[i]):
                if true_sorted[j] > 1.0 / n:
                    assert vals[i][j] >= 0.5 * truth[i][v]
                    assert truth[i][v] >= 0.5 * true_sorted[j]


def test_autotuner_and_launch_shapes_do_not_change_results(rmat14):
    """fora_graph_autotune picks spread_width / walk_blocks by measured phase times; any
    launch shape gives the same walk counts (same residues) and top-k up to the push
    rounding."""
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 12, 4444)
    p = fora.Params.make(k=50, seed=8)
    ref_ids, ref_vals, ref_st, ref = run_debug(g, sources, p)
    choice = g.autotune(sources, p)
    assert choice["spread_width"] in (1, 2, 4, 8, 16) and choice["walk_blocks"] in (3, 4, 5)
    assert choice["pipeline"] == 1  # 12 sources: too few to split
    assert choice["spread_hot"] in (0, 1) and g.tuning("spread_hot") == choice["spread_hot"]
    assert g.tuning("walk_blocks") == choice["walk_blocks"]
    for sw, wb in [(1, 3), (16, 5), (3, 4), (choice["spread_width"], choice["walk_blocks"])]:
        g.tune("spread_width", sw)
        g.tune("walk_blocks", wb)
        ids, vals, st, out = run_debug(g, sources, p, given=(ref["reserve"], ref["residue"]))
        np.testing.assert_array_equal(out["count"], ref["count"])
        np.testing.assert_array_equal(ids, ref_ids)
        _, vals2, st2, out2 = run_debug(g, sources, p)
        np.testing.assert_allclose(out2["reserve"], ref["reserve"], rtol=0, atol=ATOL_PUSH)
        assert [s.pushes for s in st2] == [s.pushes for s in ref_st]
    with pytest.raises(fora.FORAError):
        g.tune("walk_blocks", 6)
    g.tune("spread_width", 1)
    g.tune("walk_blocks", 4)
    g.tune("spread_hot", 1)


def test_host_driven_push_loop_matches_oracle(rmat14):
    """push_host_loop=1 launches the same round kernels from the host: same rounds and
    pushes as the oracle, reserve and residue within the push tolerance."""
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 5, 5151)
    p = fora.Params.make(k=50, seed=9)
    rmax = g.resolve(p)[0]
    g.tune("push_host_loop", 1)
    try:
        _, _, st, out = run_debug(g, sources, p)
        g.tune("spread_hot", 0)
        _, _, st0, out0 = run_debug(g, sources, p)
    finally:
        g.tune("push_host_loop", 0)
        g.tune("spread_hot", 1)
    np.testing.assert_allclose(out0["reserve"], out["reserve"], rtol=0, atol=ATOL_PUSH)
    assert [x.pushes for x in st0] == [x.pushes for x in st]
    for i, s in enumerate(sources):
        res_o, r_o, pst = oracle.forward_push(rp, col, int(s), 0.2, rmax)
        np.testing.assert_allclose(out["reserve"][i], res_o, rtol=0, atol=ATOL_PUSH)
        np.testing.assert_allclose(out["residue"][i], r_o, rtol=0, atol=ATOL_PUSH)
        assert st[i].pushes == pst.pushes and st[i].push_rounds == pst.rounds
    with pytest.raises(fora.FORAError):
        g.tune("push_host_loop", 2)
    with pytest.raises(fora.FORAError):
        g.tune("spread_hot", 2)


def test_device_frontier_test_equals_fp64_comparison():
    """The take decides r > RN(r_max * d) mostly in FP32 from the bit pattern of r; on
    values at, next to and around the threshold (within 2^-22 ... 2^-17 of it, where the
    FP32 band ends), at zero, denormal and FP32-underflow residues, and for r_max outside
    the FP32 fast range, the result must equal the plain FP64 comparison."""
    rng = np.random.default_rng(77)
    rmaxes = [1.9e-8, 0.1234, 3e-30, 1e-200, 2.0 ** -100, 2.0 ** -99, 1e20, 0.75, 4.2e-13]
    degs = [1, 2, 3, 16, 255, 256, 257, 1000, 2 ** 23 + 1, 2 ** 24 + 3, 2 ** 31 + 5]
    R, RM, D = [], [], []
    for rm in rmaxes:
        for d in degs:
            T = rm * float(d)
            cand = [T, 0.0, 5e-324, 2.0 ** -126, 2.0 ** -127, np.nextafter(2.0 ** -126, 0), 1.0,
                    2.0 * T, 0.5 * T]
            x = T
            for _ in range(3):
                x = np.nextafter(x, np.inf)
                cand.append(x)
            x = T
            for _ in range(3):
                x = np.nextafter(x, 0.0)
                cand.append(x)
            for e in (17, 18, 19, 20, 21, 22, 23, 24):
                cand += [T * (1 + 2.0 ** -e), T * (1 - 2.0 ** -e)]
            cand += list(T * (1 + rng.uniform(-2.0 ** -17, 2.0 ** -17, 200)))
            cand = [c for c in cand if np.isfinite(c) and c >= 0]
            R += cand
            RM += [rm] * len(cand)
            D += [d] * len(cand)
    R, RM, D = np.array(R), np.array(RM), np.array(D, dtype=np.uint32)
    want = R > RM * D.astype(np.float64)
    got = fora.threshold(R, RM, D)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, [(R[i], RM[i], D[i], got[i]) for i in bad[:5]]
    assert want.any() and (~want).any()


def test_pipelined_batch_equals_one_part(rmat14):
    """pipeline=2 and 3 (parts on their own streams, pushes staggered) give the same walk
    counts and top-k as one part, source by source (same Philox counters)."""
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 100, 6161)
    p = fora.Params.make(k=50, seed=10)
    ids1, vals1, st1 = g.ssppr_batch(sources, p)
    try:
        for parts in (2, 3):
            g.tune("pipeline", parts)
            ids2, vals2, st2 = g.ssppr_batch(sources, p)
            assert [s.walks for s in st2] == [s.walks for s in st1]
            assert [s.pushes for s in st2] == [s.pushes for s in st1]
            np.testing.assert_allclose(vals2, vals1, rtol=0, atol=ATOL_PUSH)
            # ids may differ only where the two estimates at that rank are equal within the
            # push tolerance (two near-equal nodes swapping places)
            differ = ids2 != ids1
            assert np.all(np.abs(vals2[differ] - vals1[differ]) <= 2 * ATOL_PUSH)
    finally:
        g.tune("pipeline", 1)
    with pytest.raises(fora.FORAError):
        g.tune("pipeline", 5)


@pytest.mark.parametrize("zero_hop", [False, True])
def test_rejected_neighbour_draws_follow_the_word_stream(zero_hop):
    """Lemire's method rejects a neighbour try when its low word is below 2^32 mod d, so a
    walk whose try is rejected takes an extra word and leaves the kernel's one-block-per-
    iteration alignment (it is finished word by word).  A hub with d = 100000 out-edges
    (2^32 mod d = 67296) and 100000 leaves that point back to it: every second move draws
    at the hub, about 1.6e-5 of those tries are rejected and 2.3e-5 take the careful path,
    so the ~1.1e7 Monte-Carlo walks from the hub (r_max = 1: no push) meet both about a
    hundred times or more.  Counts and weights must still equal the oracle's bit for bit."""
    hub, leaves = 0, 100000
    edges = [(hub, u) for u in range(1, leaves + 1)] + [(u, hub) for u in range(1, leaves + 1)]
    rp, col = inputs.csr_from_edges(leaves + 1, edges)
    g = fora.Graph(rp, col)
    flags = fora.FORA_ZERO_HOP if zero_hop else 0
    p = fora.Params.make(k=50, rmax=1.0, delta=1e-5, pf=1e-5, seed=99, flags=flags)
    q = oracle.ssppr(rp, col, hub, k=50, rmax=1.0, delta=1e-5, pf=1e-5, seed=99,
                     zero_hop=zero_hop)
    assert q.walk.walks > 5_000_000
    ids, vals, st, out = run_debug(g, [hub], p, given=(q.reserve[None], q.residue[None]))
    np.testing.assert_array_equal(out["count"][0], q.count)
    np.testing.assert_array_equal(out["acc"][0], q.acc)
    np.testing.assert_array_equal(ids[0], q.ids)
    assert st[0].walk_steps == q.walk.walk_steps
    g.close()

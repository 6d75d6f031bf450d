"""The balanced push (Section 4.2, Alg. 3) on the GPU against the oracle (needs a GPU).

Reserves and residues within 1e-12 (FP64 atomics reorder sums), the same node pushes,
edge pushes, push rounds and final threshold per source, and the whole balanced query
eps-accurate against power iteration."""
import numpy as np
import pytest

import inputs
import oracle
from oracle import exact

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1908_10583_gb300 as fora  # noqa: E402
from paper_1908_10583_gb300 import build as fbuild  # noqa: E402
from tests.test_gpu_parity import run_debug  # noqa: E402

ATOL_PUSH = 1e-12
COSTS = (1.0, 0.5, 5.0)  # per edge push, per node push, per walk (a walk costs ~5 edge pushes)


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


def balanced_debug(g, sources, p, costs):
    S, n = len(sources), g.n
    dbg = dict(reserve=torch.zeros((S, n), dtype=torch.float64, device="cuda"),
               residue=torch.zeros((S, n), dtype=torch.float64, device="cuda"),
               estimate=torch.zeros((S, n), dtype=torch.float64, device="cuda"))
    ids, vals, st = g.ssppr_batch_debug(sources, p, dbg, balance=costs)
    torch.cuda.synchronize()
    return ids, vals, st, {k: v.cpu().numpy() for k, v in dbg.items()}


@pytest.mark.parametrize("zero_hop", [False, True])
@pytest.mark.parametrize("costs", [COSTS, (1.0, 0.0, 0.5), (0.2, 1.0, 40.0)])
def test_balanced_push_matches_oracle(rmat14, zero_hop, costs):
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 10, inputs.SOURCE_SEED)
    flags = fora.FORA_ZERO_HOP if zero_hop else 0
    p = fora.Params.make(k=50, seed=inputs.WALK_SEED, flags=flags)
    C = g.resolve(p)[1]
    Cp = (1.0 - 0.2) * C if zero_hop else C
    ids, vals, st, out = balanced_debug(g, sources, p, costs)
    pushed = 0
    for i, s in enumerate(sources):
        res, r, pst, theta = oracle.forward_push_balanced(rp, col, s, 0.2, Cp, *costs)
        np.testing.assert_allclose(out["reserve"][i], res, rtol=0, atol=ATOL_PUSH)
        np.testing.assert_allclose(out["residue"][i], r, rtol=0, atol=ATOL_PUSH)
        assert (st[i].pushes, st[i].edge_pushes, st[i].push_rounds) == \
            (pst.pushes, pst.edge_pushes, pst.rounds)
        assert st[i].rmax == theta
        pushed += pst.pushes
    assert pushed > 10  # the cost rule let the push run


def test_free_walks_give_monte_carlo(rmat14):
    """Walk cost 0: no push at all, threshold 1 reported, and the walk phase equals the
    plain query with r_max = 1 (Monte-Carlo from the source) walk for walk."""
    rp, col, g = rmat14
    sources = inputs.uniform_sources(g.n, 4, 3)
    p = fora.Params.make(k=20, seed=5)
    _, vals_b, st_b = g.ssppr_batch_balanced(sources, p, (1.0, 1.0, 0.0))
    pm = fora.Params.make(k=20, seed=5, rmax=1.0)
    _, vals_m, st_m = g.ssppr_batch(sources, pm)
    assert all(s.pushes == 0 and s.rmax == 1.0 for s in st_b)
    assert [s.walks for s in st_b] == [s.walks for s in st_m]
    np.testing.assert_array_equal(vals_b, vals_m)


def test_balanced_queries_are_eps_accurate_and_batch_equals_single(rmat14):
    rp, col, g = rmat14
    n = len(rp) - 1
    sources = inputs.uniform_sources(n, 8, 42)
    p = fora.Params.make(k=50, seed=9)
    ids, vals, st, out = balanced_debug(g, sources, p, COSTS)
    truth = exact.power_iteration(rp, col, 0.2, sources)
    for i in range(len(sources)):
        big = truth[i] >= 1.0 / n
        assert (np.abs(out["estimate"][i][big] - truth[i][big]) / truth[i][big]).max() <= 0.5
        _, vals1, st1 = g.ssppr_batch_balanced([sources[i]], p, COSTS)
        np.testing.assert_allclose(vals1[0], vals[i], rtol=0, atol=ATOL_PUSH)
        assert st1[0].walks == st[i].walks and st1[0].rmax == st[i].rmax
    with pytest.raises(fora.FORAError):
        g.ssppr_batch_balanced(sources, p, (1.0, -1.0, 1.0))

"""Failure detection without a GPU fault (needs a GPU): every bounded device loop gives up
with an error status the host reads, allocation failures are injected on the host, and the
serving loop reports budget and wait failures.  After each failure the same graph handle
answers the next query exactly as before.  Nothing here traps, faults or hangs the device:
each failing loop has a cap that the kernel checks before it moves on."""
import numpy as np
import pytest

import inputs
import oracle

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
def small():
    rp, col = inputs.rmat_csr(12, 8, 1)
    return rp, col, fora.Graph(rp, col)


def assert_still_answers(rp, col, g, source=17):
    """The handle still gives the oracle's walk counts and top-k on a normal query."""
    p = fora.Params.make(k=20, seed=inputs.WALK_SEED)
    q = oracle.ssppr(rp, col, source, k=20, seed=inputs.WALK_SEED)
    ids, vals, st = g.ssppr(source, p)
    assert st.walks == q.walk.walks
    np.testing.assert_allclose(vals, q.vals, rtol=0, atol=1e-12)


def test_walk_cap_returns_walk_cap(small):
    """alpha = 1e-9 (stop threshold floor(alpha 2^32) = 4): every walk runs into the
    16384-move cap, and the walk kernel reports FORA_ERR_WALK_CAP instead of looping on.
    r_max = 1 leaves r(s) = 1 unpushed, and eps = 2, delta = p_f = 1/2 keep it to
    ceil(C) = 3 walks."""
    rp, col, g = small
    p = fora.Params.make(alpha=1e-9, eps=2.0, delta=0.5, pf=0.5, rmax=1.0, k=5)
    rmax, C, t_alpha = g.resolve(p)
    assert t_alpha == 4 and np.ceil(C) == 3
    with pytest.raises(fora.FORAError) as e:
        g.ssppr(5, p)
    assert e.value.code == fora.FORA_ERR_WALK_CAP
    assert_still_answers(rp, col, g)


def test_walk_overflow_is_refused_before_any_walk(small):
    """eps = 1e-3, delta = 1e-4: omega = C = (2 eps / 3 + 2) ln(2 / p_f) / (eps^2 delta)
    is about 2.8e10 walks for r(s) = 1, beyond the 2^32 a source may take."""
    rp, col, g = small
    p = fora.Params.make(eps=1e-3, delta=1e-4, pf=0.5, rmax=1.0, k=5)
    assert g.resolve(p)[1] > 2.0 ** 32
    with pytest.raises(fora.FORAError) as e:
        g.ssppr(5, p)
    assert e.value.code == fora.FORA_ERR_WALK_OVERFLOW
    assert_still_answers(rp, col, g)


@pytest.mark.parametrize("host_loop", [0, 1])
def test_push_round_cap_returns_not_converged(small, host_loop):
    """With the round cap tuned down to 2, a query whose push needs more rounds stops at
    the cap and reports FORA_ERR_PUSH_NOT_CONVERGED (device-side loop and host loop)."""
    rp, col, g = small
    p = fora.Params.make(k=20, seed=inputs.WALK_SEED)
    q = oracle.ssppr(rp, col, 17, k=20, seed=inputs.WALK_SEED)
    assert q.push.rounds > 2
    g.tune("push_host_loop", host_loop)
    g.tune("max_push_rounds", 2)
    try:
        assert g.tuning("max_push_rounds") == 2
        with pytest.raises(fora.FORAError) as e:
            g.ssppr(17, p)
        assert e.value.code == fora.FORA_ERR_PUSH_NOT_CONVERGED
        g.tune("max_push_rounds", q.push.rounds)  # exactly enough rounds
        g.ssppr(17, p)
    finally:
        g.tune("max_push_rounds", 100000)
        g.tune("push_host_loop", 0)
    with pytest.raises(fora.FORAError):
        g.tune("max_push_rounds", 0)
    assert_still_answers(rp, col, g)


def test_injected_allocation_failure_leaves_the_graph_usable(small):
    """The third device allocation of a workspace resize fails: the batched query returns
    FORA_ERR_OOM, and the next call (injection off) allocates again and answers exactly."""
    rp, col, g = small
    p = fora.Params.make(k=20, seed=inputs.WALK_SEED)
    src = inputs.uniform_sources(g.n, 40, 99)
    ids_a, vals_a, st_a = g.ssppr_batch(src[:4], p)
    fora.debug_fail_alloc(3)
    try:
        with pytest.raises(fora.FORAError) as e:
            g.ssppr_batch(src, p)   # 40 sources: the workspace grows
        assert e.value.code == fora.FORA_ERR_OOM
    finally:
        fora.debug_fail_alloc(0)
    ids_b, vals_b, st_b = g.ssppr_batch(src, p)
    np.testing.assert_array_equal(ids_b[:4], ids_a)
    np.testing.assert_allclose(vals_b[:4], vals_a, rtol=0, atol=1e-12)
    assert_still_answers(rp, col, g)


def test_injected_allocation_failure_in_graph_creation():
    rp, col = inputs.rmat_csr(10, 4, 3)
    fora.debug_fail_alloc(2)
    try:
        with pytest.raises(fora.FORAError) as e:
            fora.Graph(rp, col)
        assert e.value.code == fora.FORA_ERR_OOM
    finally:
        fora.debug_fail_alloc(0)
    g = fora.Graph(rp, col)
    assert_still_answers(rp, col, g, source=3)
    g.close()


def test_server_refuses_a_budget_below_one_query(small):
    rp, col, g = small
    one = fora.workspace_bytes(rp, 1)
    with pytest.raises(fora.FORAError) as e:
        fora.Server([g], lanes_per_graph=1, max_batch=4, memory_budget_bytes=one - 1)
    assert e.value.code == fora.FORA_ERR_OOM
    s = fora.Server([g], lanes_per_graph=1, max_batch=4, memory_budget_bytes=one)
    assert s.lane_capacity(0) == (0, 1)
    s.close()


def test_server_wait_times_out_and_the_request_still_completes(small):
    """A request that cannot finish in time: the wait returns FORA_ERR_TIMEOUT and the
    request stays queued; a later wait gets the same answer as the query alone."""
    rp, col, g = small
    s = fora.Server([g], lanes_per_graph=1, max_batch=64, memory_budget_bytes=1 << 30,
                    batch_window_ms=400.0)
    p = fora.Params.make(k=20, seed=inputs.WALK_SEED)
    t = s.submit(0, 17, p)
    with pytest.raises(fora.FORAError) as e:
        s.wait(t, 20, timeout_ms=1.0)
    assert e.value.code == fora.FORA_ERR_TIMEOUT
    ids, vals, info = s.wait(t, 20, timeout_ms=60000.0)
    ids1, vals1, _ = g.ssppr(17, p)
    np.testing.assert_allclose(vals, vals1, rtol=0, atol=1e-12)
    s.close()

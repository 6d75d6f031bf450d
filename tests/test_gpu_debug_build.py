"""The FORA_DEBUG build on the GPU (needs a GPU): with every device index check compiled in,
queries on valid inputs report no failed check and give the same results as the oracle.
The checks run in a child process that loads the debug library (FORA_LIB_DEBUG=1)."""
import os
import subprocess
import sys

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_checks():
    """Push, walk phase (plain, zero-hop), balanced push and top-k through the debug
    library against the oracle."""
    import paper_1908_10583_gb300 as fora
    from tests.test_gpu_parity import run_debug
    assert fora.load().fora_debug_checks() == 1
    rp, col = inputs.rmat_csr(14, 8, 1)
    n = len(rp) - 1
    g = fora.Graph(rp, col)
    sources = inputs.uniform_sources(n, 6, inputs.SOURCE_SEED)
    for zh in (False, True):
        p = fora.Params.make(k=50, seed=inputs.WALK_SEED, flags=fora.FORA_ZERO_HOP if zh else 0)
        qs = [oracle.ssppr(rp, col, s, k=50, seed=inputs.WALK_SEED, zero_hop=zh) for s in sources]
        ids, vals, st, out = run_debug(g, sources, p)
        for i, q in enumerate(qs):
            np.testing.assert_allclose(out["reserve"][i], q.reserve, rtol=0, atol=1e-12)
            assert st[i].pushes == q.push.pushes
        given = (np.stack([q.reserve for q in qs]), np.stack([q.residue for q in qs]))
        ids, vals, st, out = run_debug(g, sources, p, given=given)
        for i, q in enumerate(qs):
            np.testing.assert_array_equal(out["count"][i], q.count)
            np.testing.assert_array_equal(ids[i], q.ids)
    p = fora.Params.make(k=50, seed=3)
    C = g.resolve(p)[1]
    _, _, st = g.ssppr_batch_balanced(sources, p, (1.0, 0.5, 5.0))
    for i, s in enumerate(sources):
        _, _, pst, theta = oracle.forward_push_balanced(rp, col, s, 0.2, C, 1.0, 0.5, 5.0)
        assert st[i].pushes == pst.pushes and st[i].rmax == theta
    g.close()


def test_debug_build_reports_no_failed_check_and_matches_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_10583_gb300 import build as fbuild
    fbuild.build(debug=True)
    env = dict(os.environ, FORA_LIB_DEBUG="1")
    res = subprocess.run([sys.executable, "-c",
                          "import tests.test_gpu_debug_build as t; t.run_checks()"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]

"""Host arithmetic of the learned-r_max pipeline (no GPU): the cost calibration by
non-negative least squares, the modelled cost, and the label of each source (the
log2 multiplier minimising its modelled cost, refined by a parabola)."""
import numpy as np
import pytest

from paper_1908_10583_gb300 import learned_rmax as lr

pytest.importorskip("scipy")


def _runs(coef, fixed_push, fixed_walk, count=60, seed=1):
    rng = np.random.default_rng(seed)
    runs = []
    for _ in range(count):
        r = {"edge_pushes": rng.uniform(1e8, 1e10), "pushes": rng.uniform(1e6, 1e8),
             "push_rounds": rng.uniform(10, 500), "walks": rng.uniform(1e8, 1e10),
             "walk_steps": rng.uniform(4e8, 4e10), "residual_nodes": rng.uniform(1e5, 1e7)}
        r["ms_push"] = (coef["edge_push"] * r["edge_pushes"] + coef["push"] * r["pushes"]
                        + coef["push_round"] * r["push_rounds"] + fixed_push)
        r["ms_walk"] = (coef["walk"] * r["walks"] + coef["move"] * r["walk_steps"]
                        + coef["residual"] * r["residual_nodes"] + fixed_walk)
        runs.append(r)
    return runs


def test_calibration_recovers_per_unit_costs():
    coef = {"edge_push": 6e-9, "push": 2e-8, "push_round": 5e-3, "walk": 3e-8, "move": 1e-8,
            "residual": 6e-8}
    got = lr.calibrate(_runs(coef, 1.5, 7.0))
    for k, v in coef.items():
        assert got[k] == pytest.approx(v, rel=1e-6)
    assert got["push_fixed"] == pytest.approx(1.5, rel=1e-6)
    assert got["walk_fixed"] == pytest.approx(7.0, rel=1e-6)
    assert got["r2_push"] == pytest.approx(1.0) and got["r2_walk"] == pytest.approx(1.0)


def test_calibration_keeps_costs_non_negative():
    # a term that only adds noise must not come out negative
    coef = {"edge_push": 6e-9, "push": 0.0, "push_round": 5e-3, "walk": 3e-8, "move": 0.0,
            "residual": 6e-8}
    runs = _runs(coef, 0.0, 0.0, seed=2)
    rng = np.random.default_rng(3)
    for r in runs:
        r["ms_push"] *= 1 + 0.01 * rng.standard_normal()
        r["ms_walk"] *= 1 + 0.01 * rng.standard_normal()
    got = lr.calibrate(runs)
    assert all(got[k] >= 0.0 for k in coef) and got["push_fixed"] >= 0 and got["walk_fixed"] >= 0
    assert got["edge_push"] == pytest.approx(6e-9, rel=0.05)


def test_modelled_cost_is_the_linear_combination():
    coef = {"edge_push": 2.0, "push": 3.0, "push_round": 5.0, "walk": 7.0, "move": 11.0,
            "residual": 13.0}
    cnt = np.array([[1, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0], [1, 1, 1, 1, 1, 1.0]])
    np.testing.assert_allclose(lr.cost(cnt, coef), [2.0, 3.0, 41.0])


def test_labels_find_the_minimum_of_the_cost_curve():
    lg = np.log2(lr.MULTS)
    targets = np.array([-1.2, -0.3, 0.0, 0.77, 1.6])
    costs = (lg[None, :] - targets[:, None]) ** 2 + 3.0  # a parabola in log2(multiplier)
    np.testing.assert_allclose(lr.labels(costs), targets, atol=1e-12)
    # a minimum at either end of the grid is not extrapolated
    edge = np.vstack([np.arange(8.0), np.arange(8.0)[::-1]])
    np.testing.assert_array_equal(lr.labels(edge), [lg[0], lg[-1]])

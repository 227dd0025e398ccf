"""The oracle's grid form of the path cost (used only to time the oracle on the dense forest)
against its brute-force form: every cost term, flag and collision count equal bit for bit,
and the grid distances equal to the brute-force ones wherever those are negative."""
import numpy as np
import pytest

from helpers import endpoints


def _problem(name, K, S, n_cyl=None):
    import oracle
    from paper_2503_14160_gb300 import workloads
    crane = workloads.forestry_crane()
    sc = workloads.make_scene(workloads.WORKLOADS[name])
    if n_cyl is not None:
        near = np.argsort(np.hypot(sc.cylinders[:, 0], sc.cylinders[:, 1]), kind="stable")[:n_cyl]
        sc = workloads.Scene(sc.cylinders[near], sc.boxes)
    return oracle, oracle.Problem(crane, sc, oracle.CostParams(K=K, S=S))


@pytest.mark.parametrize("name,n_cyl,cell", [("dense_forest", 600, 0.5), ("dense_forest", 600, 1.3),
                                             ("single_small", None, 0.5)])
def test_grid_cost_equals_brute_force(name, n_cyl, cell):
    from paper_2503_14160_gb300 import workloads
    oracle, prob = _problem(name, 4, 8, n_cyl)
    q0, qd = endpoints(name)
    xi = workloads.random_candidates(q0, qd, 4, 24, seed=11).astype(np.float64)
    b = oracle.evaluate(prob, xi, q0, qd, with_distances=True)
    g = oracle.evaluate_grid(prob, xi, q0, qd, cell, with_distances=True)
    for f in ("J", "Jp", "Jc", "Jl", "length", "flag", "n_flagged"):
        np.testing.assert_array_equal(getattr(g, f), getattr(b, f), err_msg=f)
    neg = b.d < 0
    np.testing.assert_array_equal(g.d[neg], b.d[neg])
    assert np.all(g.d[~neg] >= 0)
    assert (b.d < 0).any() and (b.d > 0).any()     # both sides of contact are exercised
    if name == "dense_forest":
        assert prob.box.shape[0] > 0


def test_grid_cost_empty_scene():
    from paper_2503_14160_gb300 import workloads
    import oracle
    crane = workloads.forestry_crane()
    prob = oracle.Problem(crane, workloads.empty_scene(), oracle.CostParams(K=3, S=5))
    q0, qd = np.zeros(4), np.ones(4)
    xi = workloads.random_candidates(q0, qd, 3, 5, seed=1).astype(np.float64)
    b = oracle.evaluate(prob, xi, q0, qd)
    g = oracle.evaluate_grid(prob, xi, q0, qd, 0.5)
    np.testing.assert_array_equal(g.J, b.J)
    assert not g.flag.any()

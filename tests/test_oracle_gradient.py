"""Pin of the oracle's analytic gradient of the smooth cost against central finite
differences (h = 1e-4, FP64) of the oracle's smooth cost, with cylinders, boxes and joint
limit violations; and gradient descent lowers the cost."""
import numpy as np
import pytest

from paper_2503_14160_gb300 import workloads


def _fd(oracle, pb, x, q0, qd, h=1e-4):
    g = np.zeros_like(x)
    for f in range(x.shape[0]):
        for c in range(4):
            xp = x.copy()
            xm = x.copy()
            xp[f, c] += h
            xm[f, c] -= h
            g[f, c] = (oracle.smooth_cost(pb, xp[None], q0, qd)[0] -
                       oracle.smooth_cost(pb, xm[None], q0, qd)[0]) / (2 * h)
    return g


@pytest.mark.parametrize("with_boxes", [False, True])
def test_smooth_gradient_matches_finite_differences(oracle, crane, with_boxes):
    sc = workloads.make_scene(workloads.WORKLOADS["differentiable"])
    cyl = sc.cylinders[np.argsort(np.hypot(sc.cylinders[:, 0], sc.cylinders[:, 1]))[:150]]
    box = workloads.make_scene(workloads.WORKLOADS["dense_forest"]).boxes[:8] if with_boxes \
        else np.zeros((0, 6))
    K, S = 3, 8
    pb = oracle.Problem(crane, workloads.Scene(cyl, box), oracle.CostParams(K=K, S=S))
    q0 = np.array([1.24, -0.25, -1.95, 0.81])
    qd = np.array([0.52, -0.10, -1.16, 0.70])
    xi = workloads.random_candidates(q0, qd, K, 3, seed=9, spread=(0.6, 0.4, 0.5, 1.5))
    xi = xi.astype(np.float64)
    g = oracle.smooth_grad(pb, xi, q0, qd)
    for i in range(3):
        fd = _fd(oracle, pb, xi[i], q0, qd)
        assert np.linalg.norm(g[i] - fd) <= 1e-4 * np.linalg.norm(fd)


def test_free_space_gradient_is_path_energy(oracle, crane):
    """Without obstacles and inside the limits J_s = J_p, a quadratic: its gradient is zero
    at the least-squares optimum and linear in the control points."""
    K, S = 4, 8
    pb = oracle.Problem(crane, workloads.empty_scene(), oracle.CostParams(K=K, S=S))
    q0 = np.array([1.0, 0.2, -1.0, 0.5])
    qd = np.array([-1.0, 0.8, -2.0, 1.5])
    g = np.random.default_rng(3)
    a = workloads.straight_line_points(q0, qd, K) + 0.05 * g.normal(size=(K, 4))
    b = workloads.straight_line_points(q0, qd, K) + 0.05 * g.normal(size=(K, 4))
    ga, gb, gm = (oracle.smooth_grad(pb, x[None], q0, qd)[0] for x in (a, b, 0.5 * (a + b)))
    np.testing.assert_allclose(gm, 0.5 * (ga + gb), rtol=1e-9, atol=1e-12)


def test_polish_descends(oracle, crane):
    sc = workloads.make_scene(workloads.WORKLOADS["differentiable"])
    K, S = 3, 8
    pb = oracle.Problem(crane, workloads.Scene(sc.cylinders[:200], np.zeros((0, 6))),
                        oracle.CostParams(K=K, S=S))
    q0 = np.array([1.24, -0.25, -1.95, 0.81])
    qd = np.array([0.52, -0.10, -1.16, 0.70])
    xi = workloads.random_candidates(q0, qd, K, 2, seed=5, spread=(0.1, 0.05, 0.05, 0.1))
    x1 = oracle.polish(pb, xi, q0, qd, steps=3, alpha=1e-5)
    assert np.all(oracle.smooth_cost(pb, x1, q0, qd) < oracle.smooth_cost(pb, xi, q0, qd))

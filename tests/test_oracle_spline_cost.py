"""Pins of the oracle's B-spline and path cost (Sec. 4.1, Eq. path opt) against a library
B-spline (scipy), partition of unity, end conditions, straight-line and constant paths."""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from paper_2503_14160_gb300 import workloads


def test_basis_matches_scipy(oracle):
    """Cox-de Boor on the uniform knots t_i = i equals scipy's B-spline basis."""
    g = np.random.default_rng(0)
    for n_c in (9, 16, 24, 40):
        knots = np.arange(n_c + 4, dtype=np.float64)
        for tau in np.concatenate([g.uniform(3.0, n_c - 1e-9, 40), np.arange(3, n_c)]):
            mine = oracle.bspline_basis(n_c, tau)
            ref = np.array([BSpline(knots, np.eye(n_c)[i], 3, extrapolate=False)(tau)
                            for i in range(n_c)])
            ref = np.nan_to_num(ref)
            np.testing.assert_allclose(mine, ref, atol=1e-14)
            assert abs(mine.sum() - 1.0) < 1e-14     # partition of unity


def test_spline_matches_scipy_random_points(oracle):
    g = np.random.default_rng(1)
    n_c = 20
    P = g.normal(size=(n_c, 4))
    knots = np.arange(n_c + 4, dtype=np.float64)
    spl = BSpline(knots, P, 3)
    for tau in g.uniform(3.0, n_c, 100):
        np.testing.assert_allclose(oracle.bspline(P, tau), spl(tau), atol=1e-13)


def _control_points(q0, qd, xi):
    return np.concatenate([np.tile(q0, (4, 1)), xi, np.tile(qd, (4, 1))])


def test_end_conditions(oracle):
    """q(s=0) = q0 and q(s=1) = qd with zero first and second derivative at both ends:
    the moving spans are [4, K+7] in knot units (four copies of each end point)."""
    g = np.random.default_rng(2)
    K = 8
    q0, qd = g.normal(size=4), g.normal(size=4)
    P = _control_points(q0, qd, g.normal(size=(K, 4)))
    spl = BSpline(np.arange(K + 12, dtype=np.float64), P, 3)
    lo, hi = 4.0, K + 7.0
    np.testing.assert_allclose(oracle.bspline(P, lo), q0, atol=1e-14)
    np.testing.assert_allclose(oracle.bspline(P, hi), qd, atol=1e-14)
    for tau in (lo, hi):
        np.testing.assert_allclose(spl.derivative(1)(tau), 0.0, atol=1e-13)
        np.testing.assert_allclose(spl.derivative(2)(tau), 0.0, atol=1e-13)


def test_linear_precision(oracle):
    """Control points P_i = a + b (i - 2) reproduce the line q(tau) = a + b (tau - 3)...
    on uniform knots t_i = i a cubic B-spline with P_i = i gives tau - 2 (Greville
    abscissae (t_{i+1} + t_{i+2} + t_{i+3}) / 3 = i + 2)."""
    n_c = 15
    P = np.tile(np.arange(n_c, dtype=np.float64)[:, None], (1, 4))
    for tau in np.linspace(3.0, n_c - 1e-9, 57):
        np.testing.assert_allclose(oracle.bspline(P, tau), tau - 2.0, atol=1e-13)


def _scipy_path(q0, qd, xi, K, S):
    """The checkpoints q(s_k), k = 0..n_s, by scipy's B-spline."""
    P = _control_points(q0, qd, xi)
    spl = BSpline(np.arange(K + 12, dtype=np.float64), P, 3)
    n_s = (K + 3) * S
    tau = 4.0 + (K + 3) * (np.arange(n_s + 1) / n_s)
    return spl(tau)


def test_cost_terms_free_space_against_scipy(oracle, crane):
    """J_p, J_l and the path length from the oracle equal the sums of Eq. path opt taken
    over checkpoints evaluated by scipy (no obstacles, so J_c = 0)."""
    K, S = 6, 16
    pb = oracle.Problem(crane, workloads.empty_scene(), oracle.CostParams(K=K, S=S))
    g = np.random.default_rng(3)
    q0 = np.array([0.3, 0.2, -1.0, 0.5])
    qd = np.array([-2.0, 1.0, -2.0, 2.0])
    xi = workloads.straight_line_points(q0, qd, K)[None] + g.normal(size=(5, K, 4)) * 0.7
    c = oracle.evaluate(pb, xi, q0, qd)
    lo, hi = np.array(crane.q_min), np.array(crane.q_max)
    for i in range(5):
        Q = _scipy_path(q0, qd, xi[i], K, S)
        dq = np.diff(Q, axis=0)
        Jp = np.sum(dq ** 2)
        Jl = np.sum(np.maximum(0, Q[1:] - hi) ** 2 + np.maximum(0, lo - Q[1:]) ** 2)
        assert c.Jp[i] == pytest.approx(Jp, rel=1e-12)
        assert c.Jl[i] == pytest.approx(Jl, rel=1e-12, abs=1e-15)
        assert c.length[i] == pytest.approx(np.sum(np.linalg.norm(dq, axis=1)), rel=1e-12)
        assert c.Jc[i] == 0.0 and c.flag[i] == 0
        assert c.J[i] == pytest.approx(Jp + 100.0 * Jl, rel=1e-12)


def test_straight_line_length(oracle, crane):
    """Control points evenly spaced on the segment: the path stays on the segment and is
    monotone, so its length is |qd - q0|; inside the limits J_l = 0."""
    K, S = 8, 32
    pb = oracle.Problem(crane, workloads.empty_scene(), oracle.CostParams(K=K, S=S))
    q0 = np.array([2.0, 0.1, -2.0, 0.3])
    qd = np.array([-1.5, 1.0, -0.5, 2.2])
    xi = workloads.straight_line_points(q0, qd, K)[None]
    c = oracle.evaluate(pb, xi, q0, qd)
    assert c.length[0] == pytest.approx(np.linalg.norm(qd - q0), rel=1e-13)
    assert c.Jl[0] == 0.0 and c.Jc[0] == 0.0
    # Cauchy-Schwarz: the sum of squares of n_s increments of total length L is >= L^2/n_s
    assert c.Jp[0] >= np.linalg.norm(qd - q0) ** 2 / ((K + 3) * S) * (1 - 1e-12)


def test_constant_path_in_collision(oracle, crane):
    """Every control point at one configuration q*: no motion (J_p = L = 0), and J_c, J_l
    are n_s times the value at q* (worked out by hand for q* = 0 and one cylinder)."""
    K, S = 4, 8
    n_s = (K + 3) * S
    sc = workloads.Scene(np.array([[5.0, 0.3, 0.2, 0.0, 15.0]]), np.zeros((0, 6)))
    pb = oracle.Problem(crane, sc, oracle.CostParams(K=K, S=S))
    q = np.array([0.0, 0.0, 0.0, 0.0])
    xi = np.tile(q, (1, K, 1))
    c = oracle.evaluate(pb, xi, q, q, with_distances=True)
    pen = 0.45 - math.hypot(0.3125, 0.3)
    # q3 = 0 is above the jib limit -0.2: J_l per checkpoint = 0.2^2
    assert c.Jp[0] == 0.0 and c.length[0] == 0.0
    assert c.Jc[0] == pytest.approx(n_s * pen, rel=1e-12)
    assert c.Jl[0] == pytest.approx(n_s * 0.04, rel=1e-12)
    assert c.J[0] == pytest.approx(100 * n_s * pen + 100 * n_s * 0.04, rel=1e-12)
    assert c.flag[0] == 1 and c.n_flagged[0] == n_s
    np.testing.assert_allclose(c.d[0], -pen, rtol=1e-12)
    # distinct weights: J = J_p + w_c J_c + w_l J_l with J_c scaled by lambda_c
    pb2 = oracle.Problem(crane, sc, oracle.CostParams(K=K, S=S, w_c=3.0, w_l=7.0, lambda_c=2.0))
    c2 = oracle.evaluate(pb2, xi, q, q)
    assert c2.Jc[0] == pytest.approx(2.0 * n_s * pen, rel=1e-12)
    assert c2.J[0] == pytest.approx(3.0 * 2.0 * n_s * pen + 7.0 * n_s * 0.04, rel=1e-12)


def test_slew_only_collision_closed_form(oracle, crane):
    """A slew-only path moves every sphere on a circle about the z axis; the penetration
    of a cylinder at distance D from the axis follows from the law of cosines. J_c from
    the oracle equals the sum over checkpoints of that closed form (spline by scipy)."""
    K, S = 5, 24
    D, R = 6.0, 0.3
    phi = 0.4
    sc = workloads.Scene(np.array([[D * math.cos(phi), D * math.sin(phi), R, 0.0, 15.0]]),
                         np.zeros((0, 6)))
    pb = oracle.Problem(crane, sc, oracle.CostParams(K=K, S=S))
    q0 = np.array([-0.5, 0.3, -0.2, 0.0])
    qd = np.array([1.2, 0.3, -0.2, 0.0])
    g = np.random.default_rng(7)
    xi = workloads.straight_line_points(q0, qd, K)
    xi[:, 0] += g.normal(size=K) * 0.1
    c = oracle.evaluate(pb, xi[None], q0, qd)
    Q = _scipy_path(q0, qd, xi, K, S)
    # horizontal radii and heights of the sphere centres at the fixed (q2, q3, q4)
    c0, _, _ = oracle.fk(pb, [0.0, 0.3, -0.2, 0.0])
    rad = np.hypot(c0[:, 0], c0[:, 1])
    z = c0[:, 2]
    Jc = 0.0
    for k in range(1, Q.shape[0]):
        best = 0.0
        for s in range(12):
            dist = math.sqrt(rad[s] ** 2 + D ** 2 - 2 * rad[s] * D * math.cos(Q[k, 0] - phi))
            if z[s] >= 0.0:      # beside the cylinder: penetration R + r - dist
                best = max(best, R + 0.25 - dist)
            else:                # below the bottom cap: distance to the rim or the cap
                a, b = dist - R, -z[s]
                d = math.hypot(max(a, 0.0), b) if a > 0 else b
                best = max(best, 0.25 - d)
        Jc += best
    assert c.Jc[0] > 0.1
    assert c.Jc[0] == pytest.approx(Jc, rel=1e-10)


def test_smooth_penalty_limits_and_sum(oracle, crane):
    """The softplus penalty beta * softplus((m - sd) / beta) tends to max(0, m - sd) away
    from sd = m (error below beta * e^{-|m - sd| / beta}) and is summed over every
    sphere-obstacle pair and every checkpoint k = 1..n_s."""
    K, S = 4, 8
    n_s = (K + 3) * S
    beta, margin = 0.01, 0.05
    q = np.array([0.0, 0.0, 0.0, 0.0])
    xi = np.tile(q, (1, K, 1))
    # one cylinder far from everything except the jib sphere at x = 5.3125 (hand-checked:
    # the next nearest sphere is 0.87 m further away, far beyond the softplus tail)
    sc = workloads.Scene(np.array([[5.0, 0.3, 0.2, 0.0, 15.0]]), np.zeros((0, 6)))
    pb = oracle.Problem(crane, sc, oracle.CostParams(K=K, S=S, w_c=1.0, w_l=0.0,
                                                     margin=margin, beta=beta))
    J = oracle.smooth_cost(pb, xi, q, q)[0]
    sd = math.hypot(0.3125, 0.3) - 0.45          # penetrating by 0.0168 m
    x = (margin - sd) / beta                      # 6.7: on the linear branch
    # beta softplus(x) - beta x lies in (0, beta e^{-x}]; the other spheres are at least
    # 0.1875 m from the surface, adding less than beta e^{-13.7} each
    excess = J - n_s * (margin - sd)
    assert 0.0 < excess <= n_s * beta * (math.exp(-x) + 12 * math.exp(-13.7))
    assert excess == pytest.approx(n_s * beta * math.log1p(math.exp(-x)), rel=1e-3)
    # far away: the penalty vanishes
    far = workloads.Scene(np.array([[-30.0, 0.0, 0.2, 0.0, 15.0]]), np.zeros((0, 6)))
    pbf = oracle.Problem(crane, far, oracle.CostParams(K=K, S=S, w_c=1.0, w_l=0.0,
                                                       margin=margin, beta=beta))
    assert oracle.smooth_cost(pbf, xi, q, q)[0] < 1e-300 * n_s + 1e-200
    # two identical cylinders double the penalty (sum over pairs, not a minimum)
    two = workloads.Scene(np.array([[5.0, 0.3, 0.2, 0.0, 15.0]] * 2), np.zeros((0, 6)))
    pb2 = oracle.Problem(crane, two, oracle.CostParams(K=K, S=S, w_c=1.0, w_l=0.0,
                                                       margin=margin, beta=beta))
    assert oracle.smooth_cost(pb2, xi, q, q)[0] == pytest.approx(2 * J, rel=1e-12)

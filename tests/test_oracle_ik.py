"""Pins of the oracle's collision-free IK (Sec. 3.2, Eq. IK opt): the residual against the
kinematics it is made of, its Jacobian against central differences, the yaw wrap, the
damped Gauss-Newton steps against their defining properties (monotone cost, quadratic
convergence to an exact solution), and the collision term pushing a configuration out of
an obstacle."""
import math

import numpy as np
import pytest

from helpers import ROOT  # noqa: F401  (puts the oracle on sys.path)


@pytest.fixture(scope="module")
def env():
    import oracle
    from paper_2503_14160_gb300 import workloads
    crane = workloads.forestry_crane()
    return oracle, crane, workloads


def _problem(oracle, crane, cylinders=None):
    from paper_2503_14160_gb300 import workloads
    cyl = np.zeros((0, 5)) if cylinders is None else np.asarray(cylinders, dtype=np.float64)
    return oracle.Problem(crane, workloads.Scene(cyl, np.zeros((0, 6))), oracle.CostParams(K=1, S=1))


def test_residual_is_grapple_offset_and_yaw(env):
    oracle, crane, _ = env
    pb = _problem(oracle, crane)
    ik = oracle.IKParams(lambda_q=2.0, grapple_len=1.0)
    q = np.array([0.3, 0.2, -0.9, 0.8])
    _, _, T = oracle.fk(pb, q)
    target = np.array([1.0, -2.0, 0.5, -0.4])
    r, _ = oracle.ik_residual(pb, q, target, ik)
    np.testing.assert_allclose(r[:3], [T[0] - 1.0, T[1] + 2.0, T[2] - 1.0 - 0.5], atol=1e-14)
    assert r[3] == pytest.approx(2.0 * (0.3 + 0.4), abs=1e-14)
    assert r[4] == 0.0
    # the grapple centre is the lower grapple sphere of the model (T - 1.0 z)
    c, _, _ = oracle.fk(pb, q)
    np.testing.assert_allclose(c[11], [T[0], T[1], T[2] - 1.0], atol=1e-14)


@pytest.mark.parametrize("dq,want", [(1.5 * math.pi, -0.5 * math.pi), (-1.25 * math.pi, 0.75 * math.pi),
                                     (0.1, 0.1), (2.0 * math.pi + 0.2, 0.2)])
def test_yaw_residual_wraps(env, dq, want):
    oracle, crane, _ = env
    pb = _problem(oracle, crane)
    ik = oracle.IKParams()
    q = np.array([0.5, 0.3, -1.0, 0.5])
    r, _ = oracle.ik_residual(pb, q, np.array([0.0, 0.0, 0.0, 0.5 - dq]), ik)
    assert r[3] == pytest.approx(want, abs=1e-12)


@pytest.mark.parametrize("case", range(6))
def test_jacobian_matches_central_differences(env, case):
    oracle, crane, _ = env
    g = np.random.default_rng(case)
    cyl = [[3.0, 0.5, 0.4, 0.0, 15.0], [-2.5, 2.0, 0.3, 0.0, 15.0]]
    pb = _problem(oracle, crane, cyl)
    ik = oracle.IKParams(lambda_q=0.7, lambda_c=3.0)
    target = np.array([2.0, 1.0, 0.5, 0.3])
    lo, hi = np.array(crane.q_min), np.array(crane.q_max)
    q = lo + g.random(4) * (hi - lo)
    if case >= 3:   # in collision with the first tree (the boom passes through it)
        q = np.array([math.atan2(0.5, 3.0) + 0.02 * case, 0.05, -1.0, 0.5])
    r, J = oracle.ik_residual(pb, q, target, ik)
    if case >= 3:
        assert r[4] > 0.0
    h = 1e-6
    for j in range(4):
        e = np.zeros(4)
        e[j] = h
        rp, _ = oracle.ik_residual(pb, q + e, target, ik, jacobian=False)
        rm, _ = oracle.ik_residual(pb, q - e, target, ik, jacobian=False)
        np.testing.assert_allclose(J[:, j], (rp - rm) / (2 * h), atol=2e-6, rtol=1e-6)


def test_solver_converges_quadratically_to_an_exact_solution(env):
    oracle, crane, _ = env
    pb = _problem(oracle, crane)
    ik = oracle.IKParams()
    q_true = np.array([0.7, 0.4, -1.0, 1.2])
    _, _, T = oracle.fk(pb, q_true)
    target = np.array([T[0], T[1], T[2] - 1.0, 0.7])
    q, f, hist = oracle.ik_solve(pb, target, q_true + np.array([0.1, -0.05, 0.1, 0.2]), 30, ik)
    assert f < 1e-24
    assert all(b <= a for a, b in zip(hist, hist[1:]))           # accepted steps only lower it
    first = [h for h in hist if h > 0]
    assert first[2] < first[1] ** 1.5                             # faster than linear
    _, _, T2 = oracle.fk(pb, q)
    np.testing.assert_allclose([T2[0], T2[1], T2[2] - 1.0], target[:3], atol=1e-11)


def test_starts_are_philox_uniforms_in_the_limits(env):
    oracle, crane, _ = env
    pb = _problem(oracle, crane)
    ik = oracle.IKParams(seed=123)
    lo, hi = np.array(crane.q_min), np.array(crane.q_max)
    starts = np.array([oracle.ik_start(pb, ik, t, s) for t in range(40) for s in range(25)])
    assert np.all(starts >= lo) and np.all(starts < hi)
    u = (starts - lo) / (hi - lo)
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01
    w = oracle.philox4x32_10(np.array([[3, 7, oracle.IK_TAG, 0]], dtype=np.uint32), (123, 0))[0]
    np.testing.assert_array_equal(oracle.ik_start(pb, ik, 7, 3), lo + (w >> 8) * 2.0 ** -24 * (hi - lo))


def test_best_of_restarts_reaches_reachable_targets(env):
    oracle, crane, _ = env
    pb = _problem(oracle, crane)
    ik = oracle.IKParams(seed=5)
    g = np.random.default_rng(11)
    lo, hi = np.array(crane.q_min), np.array(crane.q_max)
    for t in range(5):
        q_true = lo + (0.1 + 0.8 * g.random(4)) * (hi - lo)
        _, _, T = oracle.fk(pb, q_true)
        target = np.array([T[0], T[1], T[2] - 1.0, q_true[0]])
        q, f, s = oracle.ik_solve_best(pb, target, t, 8, 60, ik)
        assert f < 1e-20, (t, f)


def test_collision_term_moves_the_crane_out_of_a_tree(env):
    """One tree on the straight line to the target: the best solution ends outside it."""
    oracle, crane, _ = env
    q_true = np.array([0.0, 0.25, -0.6, 0.5])
    pb0 = _problem(oracle, crane)
    _, _, T = oracle.fk(pb0, q_true)
    target = np.array([T[0], T[1], T[2] - 1.0, 0.0])
    # a thin tree 0.2 m beside the third boom sphere at this configuration; the grapple
    # target stays free, and raising the boom to about 0.6 rad clears the tree
    pb = _problem(oracle, crane, [[2.42, 0.2, 0.15, 0.0, 15.0]])
    assert oracle.signed_distance(pb, q_true)[0] == pytest.approx(-0.2, abs=1e-3)
    ik = oracle.IKParams(lambda_c=10.0, seed=2)
    q, f, s = oracle.ik_solve_best(pb, target, 0, 16, 80, ik)
    r, _ = oracle.ik_residual(pb, q, target, ik)
    assert oracle.signed_distance(pb, q)[0] > -1e-6
    assert np.linalg.norm(r[:3]) < 1e-3

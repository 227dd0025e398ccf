"""Pins of the trajectory-optimisation oracle (Sec. 4.2, Eq. discrete) against things other
than itself: the tip acceleration against second differences of the C oracle's forward
kinematics; the swing dynamics against the physics of a pendulum (rest, energy with a fixed
pivot, small-oscillation period, steady tilt under a constant pivot acceleration); the
collocation solver against scipy's SLSQP on the same constrained problem, and its solution's
feasibility."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def parts():
    import oracle
    import trajopt
    from paper_2503_14160_gb300 import workloads
    return oracle, trajopt, workloads.forestry_crane()


def test_tip_position_and_acceleration_follow_the_fk(parts):
    oracle, t, crane = parts
    import ctypes  # noqa: F401  (the C oracle is loaded through oracle.lib())
    prob = oracle.Problem(crane, __import__("paper_2503_14160_gb300.workloads", fromlist=["x"]).empty_scene(),
                          oracle.CostParams(K=1, S=1))
    g = np.random.default_rng(4)
    for _ in range(20):
        q0 = np.array([g.uniform(-3, 3), g.uniform(-0.3, 1.3), g.uniform(-2.6, -0.2), g.uniform(0, 2.5)])
        v, a = g.normal(size=4) * 0.4, g.normal(size=4) * 0.3
        np.testing.assert_allclose(t.tip_position(crane, q0), oracle.fk_tips(prob, q0[None])[0], atol=1e-12)
        dt = 1e-3
        qs = np.stack([q0 + v * s + 0.5 * a * s * s for s in (-dt, 0.0, dt)])
        T = oracle.fk_tips(prob, qs)
        fd = (T[2] - 2.0 * T[1] + T[0]) / (dt * dt)
        np.testing.assert_allclose(t.tip_acceleration(crane, q0, v, a), fd, atol=2e-5)


def _rk4(f, y, dt, steps):
    out = [y]
    for _ in range(steps):
        k1 = f(y)
        k2 = f(y + 0.5 * dt * k1)
        k3 = f(y + 0.5 * dt * k2)
        k4 = f(y + dt * k3)
        y = y + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        out.append(y)
    return np.array(out)


def _swing_rhs(t, tp, tip_acc=np.zeros(3)):
    def f(y):
        a, b, da, db = y
        dda, ddb = t.swing_acceleration(tp, a, b, da, db, tip_acc)
        return np.array([da, db, dda, ddb])
    return f


def test_swing_at_rest_and_in_equilibrium(parts):
    _, t, crane = parts
    tp = t.TrajParams()
    x = np.zeros(12)
    x[:4] = [0.4, 0.5, -1.0, 1.0]
    np.testing.assert_array_equal(t.dynamics(crane, tp, x, np.zeros(4)), np.zeros(12))
    # a constant horizontal tip acceleration a tilts the grapple back to alpha = -atan(a / g)
    for acc in (0.5, -2.0):
        x = np.zeros(12)
        x[:4] = [0.0, 0.4, -0.4, 1.0]          # q1 = 0, jib horizontal: the telescope moves the tip along x
        x[4] = -math.atan(acc / t.GRAVITY)
        u = np.array([0.0, 0.0, 0.0, acc])
        np.testing.assert_allclose(t.tip_acceleration(crane, x[:4], x[6:10], u), [acc, 0, 0], atol=1e-15)
        xd = t.dynamics(crane, tp, x, u)
        assert abs(xd[10]) < 1e-14 and abs(xd[11]) < 1e-14


def test_swing_energy_is_conserved_with_a_fixed_pivot(parts):
    _, t, _ = parts
    tp = t.TrajParams()
    ell, g = tp.grapple_len, t.GRAVITY
    Y = _rk4(_swing_rhs(t, tp), np.array([0.3, 0.2, 0.0, 0.5]), 1e-3, 5000)
    a, b, da, db = Y.T
    E = 0.5 * ell * ell * (da ** 2 + np.cos(a) ** 2 * db ** 2) - g * ell * np.cos(a) * np.cos(b)
    assert np.max(np.abs(E - E[0])) < 1e-9


def test_swing_small_oscillation_period(parts):
    _, t, _ = parts
    for ell in (1.0, 2.5):
        tp = t.TrajParams(grapple_len=ell)
        dt = 1e-4
        Y = _rk4(_swing_rhs(t, tp), np.array([1e-4, 0.0, 0.0, 0.0]), dt, int(4.0 * 2 * math.pi * math.sqrt(ell / 9.81) / dt))
        a = Y[:, 0]
        up = np.nonzero((a[:-1] < 0) & (a[1:] >= 0))[0]
        times = (up + a[up] / (a[up] - a[up + 1])) * dt          # linear interpolation of the crossing
        period = np.mean(np.diff(times))
        assert period == pytest.approx(2 * math.pi * math.sqrt(ell / t.GRAVITY), rel=1e-5)


def _small_problem(t, crane, N, q0, qd):
    tp = t.TrajParams(N=N)
    s = np.linspace(0.0, 1.0, N + 1)[:, None]
    q_star = q0[None] + (3 * s ** 2 - 2 * s ** 3) * (qd - q0)[None]   # a smooth path from rest to rest
    return t.TrajProblem(crane, tp, q_star, q0, qd), tp


def test_collocation_solution_is_feasible(parts):
    _, t, crane = parts
    q0, qd = np.array([0.2, 0.3, -1.2, 0.5]), np.array([1.4, 0.6, -0.8, 1.5])
    prob, tp = _small_problem(t, crane, 10, q0, qd)
    z0 = prob.initial_guess()
    rec = []
    z, lam, _ = prob.solve(z0, record=rec)
    c = prob.constraints(z)
    assert np.max(np.abs(c)) < 2e-4
    assert np.max(np.abs(prob.violation(z))) < 1e-4
    # no joint can outrun its velocity limit over the path
    t_min = np.max(np.abs(qd - q0) / np.asarray(tp.dq_max))
    assert z[0] > t_min * (1 - 1e-3)
    # the merit never increased within an outer step, and some steps were accepted
    assert any(r[3] for r in rec)
    _, X, _ = prob.unpack(z)
    np.testing.assert_allclose(X[0, :4], q0, atol=2e-4)
    np.testing.assert_allclose(X[-1, :4], qd, atol=2e-4)


def test_collocation_matches_scipy_slsqp(parts):
    """The same constrained problem (objective of Eq. discrete, trapezoidal defects and end
    states as equalities, state bounds) solved by scipy's SLSQP from the same start reaches
    the same final time and objective."""
    _, t, crane = parts
    scipy_opt = pytest.importorskip("scipy.optimize")
    q0, qd = np.array([0.0, 0.4, -1.0, 0.8]), np.array([0.9, 0.7, -0.7, 1.4])
    prob, tp = _small_problem(t, crane, 6, q0, qd)
    prob.tp = dataclasses_replace(tp, outer=12, inner=10)
    z0 = prob.initial_guess()
    z, _, _ = prob.solve(z0)

    def objective(zz):
        _, X, U = prob.unpack(zz)
        return (zz[0] + tp.omega_s * np.sum(np.asarray(tp.R) * U[1:] ** 2)
                + tp.omega_t * np.sum((X[1:, :4] - prob.q_star[1:]) ** 2))

    lo = np.concatenate([[1e-3], np.tile(np.concatenate([prob.x_min, -1e30 * np.ones(4)]), tp.N + 1)])
    hi = np.concatenate([[1e30], np.tile(np.concatenate([prob.x_max, 1e30 * np.ones(4)]), tp.N + 1)])
    bounds = [(a if a > -1e29 else None, b if b < 1e29 else None) for a, b in zip(lo, hi)]
    res = scipy_opt.minimize(objective, z0, method="SLSQP", bounds=bounds,
                             constraints=[{"type": "eq", "fun": prob.constraints}],
                             options={"maxiter": 500, "ftol": 1e-12})
    assert res.success, res.message
    assert z[0] == pytest.approx(res.x[0], rel=2e-3)
    assert objective(z) == pytest.approx(res.fun, rel=1e-3)


def dataclasses_replace(obj, **kw):
    import dataclasses
    return dataclasses.replace(obj, **kw)

"""Parity of the batched collision-free IK (Sec. 3.2, Eq. IK opt) with the oracle.

The GPU solves in FP32 and the oracle in FP64 on the same targets and the same starting
points. The residual the kernel reports at its answer is checked against the oracle's
residual at that answer (elementwise, within the FP32 kinematics error); a single damped
Gauss-Newton step from a given start against the oracle's step; the starting points against
the oracle's Philox draws; and full solves by what they must reach (reachable targets
solved, a tree cleared). Whole solves are not compared step for step: FP32 and FP64 runs
part ways over tens of iterations, most visibly where the collision term switches on.

Tolerances:
  R_TOL   |r_gpu - r_oracle(q_gpu)| per component, in metres: the position rows carry the
          FP32 kinematics over a lever of about 10 m (a few ulp of 10 m, ~1e-6 m each); the
          collision row the distance error D_TOL times lambda_c.
  STEP    one step: |q_gpu - q_oracle| <= 2e-3 |step| + 2e-5 per joint. The FP32 normal
          equations carry ~1e-7 times the condition number of H + mu diag(H) (below 1e4
          for the starts used here) relative to the step.
"""
import math

import numpy as np
import pytest

from helpers import Setup

pytestmark = pytest.mark.gpu

R_TOL = 2e-5


@pytest.fixture(scope="module")
def lib():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


def _scene(name=None, cylinders=None):
    from paper_2503_14160_gb300 import workloads
    if name is not None:
        return workloads.make_scene(workloads.WORKLOADS[name])
    cyl = np.zeros((0, 5)) if cylinders is None else np.asarray(cylinders, dtype=np.float64)
    return workloads.Scene(cyl, np.zeros((0, 6)))


def _run(lib, s, targets, ik, q_init=None):
    import torch
    n = targets.shape[0]
    t = torch.from_numpy(np.ascontiguousarray(targets, np.float32)).cuda()
    qi = None if q_init is None else torch.from_numpy(np.ascontiguousarray(q_init, np.float32)).cuda()
    q = torch.zeros(max(n, 1), 4, dtype=torch.float32, device="cuda")
    f = torch.zeros(max(n, 1), dtype=torch.float32, device="cuda")
    k = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    r = torch.zeros(max(n, 1), 5, dtype=torch.float32, device="cuda")
    lib.cp_ik(s.h, t, n, ik, q, f, q_init=qi, restart=k, r=r)
    torch.cuda.synchronize()
    return (q.cpu().numpy()[:n].astype(np.float64), f.cpu().numpy()[:n].astype(np.float64),
            k.cpu().numpy()[:n], r.cpu().numpy()[:n].astype(np.float64))


def _oracle_ik(s, ik):
    return s.oracle.IKParams(lambda_q=ik.lambda_q, lambda_c=ik.lambda_c, grapple_len=ik.grapple_len,
                             mu0=ik.mu0, seed=ik.seed)


def _reachable(s, crane, n, seed, grapple_len, clearance=None):
    """Targets at the grapple of configurations uniform in the inner 80% of the limits
    (free of collision by `clearance` when given) and their configurations."""
    g = np.random.default_rng(seed)
    lo, hi = np.array(crane.q_min), np.array(crane.q_max)
    qs, ts = [], []
    while len(qs) < n:
        q = lo + (0.1 + 0.8 * g.random(4)) * (hi - lo)
        if clearance is not None and s.oracle.signed_distance(s.problem, q)[0] <= clearance:
            continue
        _, _, T = s.oracle.fk(s.problem, q)
        qs.append(q)
        ts.append([T[0], T[1], T[2] - grapple_len, q[0]])
    return np.array(qs), np.array(ts)


def _check_residuals(s, q, r, f, targets, oik):
    """The kernel's r and |r|^2 at its answer against the oracle's residual at that answer."""
    lam = max(1.0, oik.lambda_q, oik.lambda_c)
    for i in range(q.shape[0]):
        ro, _ = s.oracle.ik_residual(s.problem, q[i], targets[i].astype(np.float32).astype(np.float64),
                                     oik, jacobian=False)
        np.testing.assert_allclose(r[i], ro, rtol=0, atol=R_TOL * lam, err_msg=f"target {i}")
        assert abs(f[i] - float(r[i] @ r[i])) <= 1e-6 * f[i] + 1e-12


def test_starting_points_are_the_oracle_draws(lib, crane):
    """iters = 0: the answer is the start of lowest |r|^2 (12 starts: more than one per warp)."""
    s = Setup(crane, _scene("single_large"), N=4, K=2, S=2)
    try:
        ik = lib.make_ik_params(seed=77, query=3, restarts=12, iters=0, lambda_q=2.0, grapple_len=1.25)
        oik = _oracle_ik(s, ik)
        g = np.random.default_rng(5)
        targets = np.array([-9.0, -9.0, -0.5, -math.pi]) + g.random((64, 4)) * np.array([18.0, 18.0, 2.0, 2 * math.pi])
        q, f, k, r = _run(lib, s, targets, ik)
        lo, hi = np.array(crane.q_min), np.array(crane.q_max)
        tg = targets.astype(np.float32).astype(np.float64)
        for t in range(targets.shape[0]):
            starts = np.array([s.oracle.ik_start(s.problem, oik, t, j, query=3) for j in range(12)])
            assert 0 <= k[t] < 12
            assert np.all(np.abs(q[t] - starts[k[t]]) <= 1e-6 * (hi - lo)), (t, q[t], starts[k[t]])
            fo = []
            for j in range(12):
                ro, _ = s.oracle.ik_residual(s.problem, starts[j], tg[t], oik, jacobian=False)
                fo.append(float(ro @ ro))
            fo = np.array(fo)
            # the chosen start is the oracle's best up to the FP32 error of |r|^2 (twice
            # |r| times the error of r, on both sides)
            assert fo[k[t]] <= fo.min() + 4e-4 * 2.0 * math.sqrt(fo[k[t]]) + 1e-9
        _check_residuals(s, q, r, f, targets, oik)
    finally:
        s.close()


def test_warm_start_is_start_zero(lib, crane):
    s = Setup(crane, _scene(), N=4, K=2, S=2)
    try:
        ik = lib.make_ik_params(restarts=1, iters=0)
        g = np.random.default_rng(3)
        q_init = np.array(crane.q_min) + g.random((40, 4)) * (np.array(crane.q_max) - np.array(crane.q_min))
        q_init[:5] *= 1.5   # outside the limits: clipped
        targets = g.random((40, 4))
        q, f, k, r = _run(lib, s, targets, ik, q_init=q_init)
        want = np.clip(q_init.astype(np.float32), np.float32(crane.q_min), np.float32(crane.q_max))
        np.testing.assert_array_equal(q.astype(np.float32), want)
        np.testing.assert_array_equal(k, 0)
    finally:
        s.close()


@pytest.mark.parametrize("scene", ["free", "forest", "dense"])
def test_one_step_matches_the_oracle(lib, crane, scene):
    """One damped Gauss-Newton step from the same start; in the forests most starts collide,
    so the collision row and its Jacobian take part. The dense forest (5000 trees and 50
    boxes) exceeds the obstacle count the kernel stages in shared memory."""
    name = {"free": None, "forest": "single_large", "dense": "dense_forest"}[scene]
    s = Setup(crane, _scene(name), N=4, K=2, S=2)
    try:
        ik = lib.make_ik_params(restarts=1, iters=1, lambda_q=2.0, lambda_c=5.0, grapple_len=1.25,
                                mu0=1e-2)
        oik = _oracle_ik(s, ik)
        q_true, targets = _reachable(s, crane, 96, seed=21, grapple_len=1.25)
        g = np.random.default_rng(22)
        q_init = q_true + g.normal(0.0, 0.15, q_true.shape)
        q_init = np.clip(q_init, crane.q_min, crane.q_max).astype(np.float32).astype(np.float64)
        tg = targets.astype(np.float32).astype(np.float64)
        q, f, k, r = _run(lib, s, targets, ik, q_init=q_init)
        n_coll = 0
        for i in range(q.shape[0]):
            r0, _ = s.oracle.ik_residual(s.problem, q_init[i], tg[i], oik, jacobian=False)
            n_coll += r0[4] > 0
            qo, fo, _ = s.oracle.ik_solve(s.problem, tg[i], q_init[i], 1, oik)
            step = np.max(np.abs(qo - q_init[i]))
            f0 = float(r0 @ r0)
            if step == 0.0:
                # the oracle rejected its step: so must the kernel, unless the two costs
                # are within the FP32 error of each other
                if not np.array_equal(q[i], q_init[i]):
                    fn = float(np.sum(s.oracle.ik_residual(s.problem, q[i], tg[i], oik, jacobian=False)[0] ** 2))
                    assert fn >= f0 - 1e-4 * math.sqrt(f0) - 1e-9, i
                continue
            if np.array_equal(q[i], q_init[i]):
                # the kernel rejected the step the oracle took: only when the oracle's gain
                # is within the FP32 error of the cost
                assert fo >= f0 - 1e-4 * math.sqrt(f0) - 1e-9, i
                continue
            np.testing.assert_allclose(q[i], qo, rtol=0, atol=2e-3 * step + 2e-5, err_msg=f"start {i}")
        if scene != "free":
            assert n_coll >= 10
        _check_residuals(s, q, r, f, targets, oik)
    finally:
        s.close()


def test_reachable_targets_are_solved_in_free_space(lib, crane):
    s = Setup(crane, _scene(), N=4, K=2, S=2)
    try:
        ik = lib.make_ik_params(seed=5, restarts=8, iters=60)
        oik = _oracle_ik(s, ik)
        _, targets = _reachable(s, crane, 128, seed=11, grapple_len=1.0)
        q, f, k, r = _run(lib, s, targets, ik)
        _check_residuals(s, q, r, f, targets, oik)
        lo, hi = np.array(crane.q_min, np.float32), np.array(crane.q_max, np.float32)
        assert np.all(q.astype(np.float32) >= lo) and np.all(q.astype(np.float32) <= hi)
        # position within 1e-4 m and yaw within 1e-5 rad of every target
        assert np.all(np.linalg.norm(r[:, :3], axis=1) < 1e-4), np.linalg.norm(r[:, :3], axis=1).max()
        assert np.all(np.abs(r[:, 3]) < 1e-5)
        # the oracle from the same starts solves the first few as well
        for t in range(8):
            qo, fo, _ = s.oracle.ik_solve_best(s.problem, targets[t], t, 8, 60, oik)
            assert fo < 1e-16 and f[t] < 1e-8
    finally:
        s.close()


def test_collision_term_clears_a_tree(lib, crane):
    """The oracle's tree case: the straight solution passes through a thin tree; with
    lambda_c = 10 the best solution reaches the target with the boom raised clear of it."""
    s = Setup(crane, _scene(cylinders=[[2.42, 0.2, 0.15, 0.0, 15.0]]), N=4, K=2, S=2)
    try:
        q_true = np.array([0.0, 0.25, -0.6, 0.5])
        assert s.oracle.signed_distance(s.problem, q_true)[0] == pytest.approx(-0.2, abs=1e-3)
        _, _, T = s.oracle.fk(s.problem, q_true)
        targets = np.array([[T[0], T[1], T[2] - 1.0, 0.0]])
        ik = lib.make_ik_params(lambda_c=10.0, seed=2, restarts=16, iters=80)
        q, f, k, r = _run(lib, s, targets, ik)
        _check_residuals(s, q, r, f, targets, _oracle_ik(s, ik))
        assert s.oracle.signed_distance(s.problem, q[0])[0] > -1e-4
        assert np.linalg.norm(r[0, :3]) < 1e-3
    finally:
        s.close()


def grasp_targets(s, crane, n, seed, grapple_len=1.0):
    """The benchmarked grasp poses: accepted draws (collision-free by the clearance, grapple
    centre in the height band, both by the oracle), their grapple centres and slew angles."""
    from paper_2503_14160_gb300 import workloads

    def accept(q):
        zg = s.oracle.fk_tips(s.problem, q)[:, 2] - grapple_len
        return ((s.oracle.signed_distance(s.problem, q) > workloads.GRASP_CLEARANCE)
                & (zg > workloads.GRASP_Z[0]) & (zg < workloads.GRASP_Z[1]))

    q = workloads.grasp_configurations(crane, accept, n, seed=seed)
    T = s.oracle.fk_tips(s.problem, q)
    return np.column_stack([T[:, 0], T[:, 1], T[:, 2] - grapple_len, q[:, 0]])


def test_grasp_batch(lib, crane):
    """The benchmarked workload (16384 grasp poses in the 20-tree stand, 8 starts, 50
    iterations): residuals at sampled answers against the oracle, answers inside the limits,
    and the solved fraction of a sample close to the oracle's from the same starts."""
    from paper_2503_14160_gb300 import workloads
    s = Setup(crane, _scene(workloads.IK_SCENE), N=4, K=2, S=2)
    try:
        ik = lib.make_ik_params(seed=9, restarts=8, iters=50)
        oik = _oracle_ik(s, ik)
        targets = grasp_targets(s, crane, 16384, seed=1)
        q, f, k, r = _run(lib, s, targets, ik)
        lo, hi = np.array(crane.q_min, np.float32), np.array(crane.q_max, np.float32)
        assert np.all(q.astype(np.float32) >= lo) and np.all(q.astype(np.float32) <= hi)
        assert np.all((k >= 0) & (k < 8))
        assert np.all(np.isfinite(f))
        idx = np.random.default_rng(4).choice(16384, 48, replace=False)
        _check_residuals(s, q[idx], r[idx], f[idx], targets[idx], oik)
        # every target has a collision-free answer; most are found
        assert np.mean(f < 1e-6) > 0.7
        sub = idx[:24]
        tg = targets.astype(np.float32).astype(np.float64)
        solved_o = [s.oracle.ik_solve_best(s.problem, tg[t], int(t), 8, 50, oik)[1] < 1e-6 for t in sub]
        solved_g = f[sub] < 1e-6
        assert solved_g.sum() >= sum(solved_o) - 3, (solved_g.sum(), sum(solved_o))
    finally:
        s.close()


def test_forward_kinematics(lib, crane):
    """Sphere centres and tip against the oracle's kinematics, limits and beyond."""
    import torch
    s = Setup(crane, _scene(), N=4, K=2, S=2)
    try:
        g = np.random.default_rng(8)
        lo, hi = np.array(crane.q_min), np.array(crane.q_max)
        q = lo + (hi - lo) * (-0.2 + 1.4 * g.random((1000, 4)))
        q32 = q.astype(np.float32)
        qt = torch.from_numpy(q32).cuda()
        ns = len(crane.spheres)
        c = torch.zeros(1000, ns, 3, device="cuda")
        t = torch.zeros(1000, 3, device="cuda")
        lib.cp_forward_kinematics(s.h, qt, 1000, c, t)
        lib.cp_forward_kinematics(s.h, qt, 0, c, t)
        torch.cuda.synchronize()
        c, t = c.cpu().numpy(), t.cpu().numpy()
        for i in range(1000):
            co, _, To = s.oracle.fk(s.problem, q32[i].astype(np.float64))
            np.testing.assert_allclose(c[i], co, rtol=0, atol=1e-5)
            np.testing.assert_allclose(t[i], To, rtol=0, atol=1e-5)
        np.testing.assert_allclose(s.oracle.fk_tips(s.problem, q32.astype(np.float64)), t, rtol=0, atol=1e-5)
    finally:
        s.close()


def test_edge_cases(lib, crane):
    import torch
    s = Setup(crane, _scene(), N=4, K=2, S=2)
    try:
        t = torch.zeros(1, 4, device="cuda")
        q = torch.zeros(1, 4, device="cuda")
        f = torch.zeros(1, device="cuda")
        lib.cp_ik(s.h, t, 0, lib.make_ik_params(), q, f)   # empty batch: nothing launched
        for bad in (dict(restarts=0), dict(restarts=lib.CP_IK_MAX_RESTARTS + 1), dict(iters=-1),
                    dict(mu0=0.0), dict(lambda_c=-1.0)):
            with pytest.raises(Exception):
                lib.cp_ik(s.h, t, 1, lib.make_ik_params(**bad), q, f)
        with pytest.raises(Exception):
            lib.cp_ik(s.h, t, -1, lib.make_ik_params(), q, f)
        # the largest start count: 128 starts per warp
        _, targets = _reachable(s, crane, 2, seed=1, grapple_len=1.0)
        qq, ff, kk, rr = _run(lib, s, targets, lib.make_ik_params(restarts=lib.CP_IK_MAX_RESTARTS, iters=3))
        assert np.all((kk >= 0) & (kk < lib.CP_IK_MAX_RESTARTS))
        _check_residuals(s, qq, rr, ff, targets, _oracle_ik(s, lib.make_ik_params()))
    finally:
        s.close()

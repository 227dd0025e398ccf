"""GPU parity of the differentiable form: the smooth cost (softplus collision penalty at
margin 0.05 m), its adjoint kernel against the oracle's analytic FP64 gradient (itself
pinned to central differences), the torch.autograd.Function around them, and gradient
polish (plain gradient descent) against the oracle's."""
import numpy as np
import pytest

from helpers import Setup, endpoints

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


@pytest.fixture(scope="module")
def crane():
    from paper_2503_14160_gb300 import workloads
    return workloads.forestry_crane()


def _scene(n_cyl=None, boxes=False):
    from paper_2503_14160_gb300 import workloads
    sc = workloads.make_scene(workloads.WORKLOADS["differentiable"])
    cyl = sc.cylinders
    if n_cyl is not None:
        cyl = cyl[np.argsort(np.hypot(cyl[:, 0], cyl[:, 1]), kind="stable")[:n_cyl]]
    box = workloads.make_scene(workloads.WORKLOADS["dense_forest"]).boxes[:10] if boxes else sc.boxes
    return workloads.Scene(cyl, box)


def _gpu(lib, s, xi, q0, qd, grad=True):
    import torch
    lib.cp_set_endpoints(s.h, q0, qd)
    x = torch.from_numpy(np.ascontiguousarray(xi, np.float32)).cuda()
    n = xi.shape[0]
    J = torch.zeros(n, dtype=torch.float64, device="cuda")
    if not grad:
        lib.cp_smooth_cost(s.h, x, n, J)
        torch.cuda.synchronize()
        return J.cpu().numpy(), None
    d = torch.zeros_like(x)
    lib.cp_smooth_cost_grad(s.h, x, n, None, J, d)
    torch.cuda.synchronize()
    return J.cpu().numpy(), d.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("K,S,n,n_cyl,boxes", [(4, 8, 16, 200, False), (6, 13, 9, 300, True),
                                               (32, 64, 6, None, False)])
def test_smooth_cost_and_gradient(lib, crane, K, S, n, n_cyl, boxes):
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("differentiable")
    s = Setup(crane, _scene(n_cyl, boxes), N=n, K=K, S=S)
    try:
        xi = workloads.random_candidates(q0, qd, K, n, seed=K + S, spread=(0.3, 0.15, 0.2, 0.3))
        J, g = _gpu(lib, s, xi, q0, qd)
        Jo = s.oracle.smooth_cost(s.problem, xi.astype(np.float64), q0, qd)
        go = s.oracle.smooth_grad(s.problem, xi.astype(np.float64), q0, qd)
        np.testing.assert_allclose(J, Jo, rtol=1e-4)
        # forward-only entry point gives the same J
        J2, _ = _gpu(lib, s, xi, q0, qd, grad=False)
        np.testing.assert_array_equal(J2, J)
        for i in range(n):
            rel = np.linalg.norm(g[i] - go[i]) / np.linalg.norm(go[i])
            assert rel <= 1e-3, (i, rel)
    finally:
        s.close()


def test_gradient_against_central_differences(lib, crane):
    """The GPU adjoint against central differences (h = 1e-4) of the oracle's FP64 cost."""
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("differentiable")
    K, S = 3, 8
    s = Setup(crane, _scene(150), N=2, K=K, S=S)
    try:
        xi = workloads.random_candidates(q0, qd, K, 2, seed=4, spread=(0.3, 0.15, 0.2, 0.3))
        _, g = _gpu(lib, s, xi, q0, qd)
        h = 1e-4
        for i in range(2):
            fd = np.zeros((K, 4))
            for f in range(K):
                for c in range(4):
                    xp = xi[i].astype(np.float64).copy()
                    xm = xp.copy()
                    xp[f, c] += h
                    xm[f, c] -= h
                    fd[f, c] = (s.oracle.smooth_cost(s.problem, xp[None], q0, qd)[0] -
                                s.oracle.smooth_cost(s.problem, xm[None], q0, qd)[0]) / (2 * h)
            assert np.linalg.norm(g[i] - fd) / np.linalg.norm(fd) <= 1e-3
    finally:
        s.close()


def test_autograd_function(lib, crane):
    import torch
    from paper_2503_14160_gb300 import workloads
    from paper_2503_14160_gb300.autograd import path_cost
    q0, qd = endpoints("differentiable")
    s = Setup(crane, _scene(200), N=8, K=4, S=8)
    try:
        lib.cp_set_endpoints(s.h, q0, qd)
        xi = workloads.random_candidates(q0, qd, 4, 8, seed=1, spread=(0.3, 0.15, 0.2, 0.3))
        x = torch.from_numpy(xi).cuda().requires_grad_(True)
        w = torch.linspace(0.5, 2.0, 8, dtype=torch.float64, device="cuda")
        (path_cost(x, s.planner) * w).sum().backward()
        _, g = _gpu(lib, s, xi, q0, qd)
        np.testing.assert_allclose(x.grad.cpu().numpy(), g * w.cpu().numpy()[:, None, None],
                                   rtol=1e-6, atol=1e-6 * np.abs(g).max())
    finally:
        s.close()


def test_polish_matches_oracle(lib, crane):
    """Ten gradient-descent steps (alpha = 1e-3) on the best candidates of a short plan."""
    import torch
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("differentiable")
    K, S = 8, 16
    s = Setup(crane, _scene(400), N=512, K=K, S=S, seed=3)
    try:
        lib.cp_set_endpoints(s.h, q0, qd)
        lib.cp_plan(s.h, 30, K=K)
        xi = torch.zeros(512, K, 4, device="cuda")
        J = torch.zeros(512, dtype=torch.float64, device="cuda")
        lib.cp_sample(s.h, 30, xi)
        lib.cp_evaluate(s.h, xi, 512, J)
        top = torch.argsort(J)[:8]
        best = xi[top].contiguous()
        start = best.cpu().numpy().astype(np.float64)
        lib.cp_polish(s.h, best, 8, 10, 1e-3)
        torch.cuda.synchronize()
        got = best.cpu().numpy().astype(np.float64)
        want = s.oracle.polish(s.problem, start, q0, qd, 10, 1e-3)
        moved = np.linalg.norm((want - start).reshape(8, -1), axis=1)
        err = np.linalg.norm((got - want).reshape(8, -1), axis=1)
        assert np.all(err <= 1e-3 * np.maximum(moved, 1e-3) + 1e-5), (err, moved)
        Jg = s.oracle.smooth_cost(s.problem, got, q0, qd)
        J0 = s.oracle.smooth_cost(s.problem, start, q0, qd)
        assert np.all(Jg <= J0 * (1 + 1e-6))          # descent does not increase the cost here
    finally:
        s.close()

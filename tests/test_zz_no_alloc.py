"""cp_evaluate_static: candidate evaluation for callers that may not allocate GPU memory
while they run (a real-time control loop, where cudaMalloc can stall the device for an
unbounded time, or a plug-in whose host application owns all device memory). It must give
the same results as the planner's cp_evaluate, call after call, with its fixed scratch.

This file is collected last so that a run stopping at its first failure has already run
every other test."""
import numpy as np
import pytest

from helpers import D_TOL, J_REL, Setup, cost_tolerance, endpoints

pytestmark = pytest.mark.gpu


def _scene(name, n_cyl=None):
    from paper_2503_14160_gb300 import workloads
    sc = workloads.make_scene(workloads.WORKLOADS[name])
    cyl = sc.cylinders
    if n_cyl is not None:
        cyl = cyl[np.argsort(np.hypot(cyl[:, 0], cyl[:, 1]), kind="stable")[:n_cyl]]
    return workloads.Scene(cyl, sc.boxes[:20])


def _static_eval(cp, model, scene, K, S, q0, qd, xi):
    import torch
    cyl = torch.from_numpy(np.ascontiguousarray(scene.cylinders)).cuda()
    box = torch.from_numpy(np.ascontiguousarray(scene.boxes)).cuda()
    xt = torch.from_numpy(xi).cuda()
    n = xi.shape[0]
    J = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    flag = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    terms = torch.zeros(n, 5, dtype=torch.float64, device="cuda")
    cp.cp_evaluate_static(model, cyl, scene.n_cyl, box, scene.n_box, K, S, 100.0, 100.0, 1.0,
                          q0, qd, xt, n, J, flag, terms)
    torch.cuda.synchronize()
    return J.cpu().numpy(), flag.cpu().numpy(), terms.cpu().numpy()


def test_static_evaluation_matches_planner_twice():
    from paper_2503_14160_gb300 import build, craneplan as cp, workloads
    build.build()
    cp.load()
    crane = workloads.forestry_crane()
    model = cp.make_model(crane)
    cases = [("single_small", None, 8, 32, 256, 1), ("dense_forest", 300, 5, 7, 37, 2)]
    for name, n_cyl, K, S, n, seed in cases:     # two calls in a row, different sizes
        scene = _scene(name, n_cyl)
        q0, qd = endpoints(name)
        xi = workloads.random_candidates(q0, qd, K, n, seed=seed)
        Js, fs, ts = _static_eval(cp, model, scene, K, S, q0, qd, xi)
        s = Setup(crane, scene, N=n, K=K, S=S)
        try:
            g = s.evaluate(xi, q0, qd)
        finally:
            s.close()
        n_near = (g["terms"][:, 4] + 0)              # a generous count: flagged checkpoints
        tol = J_REL * np.abs(g["J"]) + 100.0 * D_TOL * (n_near + 1)
        assert np.all(np.abs(Js - g["J"]) <= tol)
        np.testing.assert_array_equal(fs, g["flag"])
        np.testing.assert_allclose(ts[:, :4], g["terms"][:, :4], rtol=J_REL, atol=1e-9)
        np.testing.assert_array_equal(ts[:, 4], g["terms"][:, 4])


def test_static_evaluation_rejects_oversize():
    import torch
    from paper_2503_14160_gb300 import build, craneplan as cp, workloads
    build.build()
    cp.load()
    model = cp.make_model(workloads.forestry_crane())
    n, K, S = 200000, 32, 128             # partial sums alone would need ~2.5 GB
    xi = torch.zeros(1, K, 4, device="cuda")
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    empty = torch.zeros(0, 5, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CranePlanError) as e:
        cp.cp_evaluate_static(model, empty, 0, empty, 0, K, S, 100.0, 100.0, 1.0,
                              np.zeros(4), np.ones(4), xi, n, J)
    assert e.value.status == -1 and "scratch" in str(e.value)

"""GPU parity of the path evaluation with the convex-hull collision model
(collision_model = CP_COLLISION_HULLS) against the oracle's evaluate_hulls: per-checkpoint
penetration within the hull tolerance (2e-5 m), collision flags wherever the oracle's depth
is above 1e-4 m, and J within 1e-4 relative plus w_c lambda_c 2e-5 per checkpoint in
contact; a plan with the hull model against the sphere-free oracle cost of its result."""
import numpy as np
import pytest

from helpers import Setup, endpoints, unpack_flags

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def lib():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


def _setup(lib, crane, name, N, K, S):
    from paper_2503_14160_gb300 import workloads
    s = Setup(crane, workloads.make_scene(workloads.WORKLOADS[name]), N=N, K=K, S=S)
    s.planner.close()
    s.planner = lib.Planner(crane, s.scene, lib.make_params(N, K, S, collision_model=lib.CP_COLLISION_HULLS))
    return s


@pytest.mark.parametrize("name,N,K,S", [("single_small", 40, 4, 16), ("single_large", 12, 5, 7)])
def test_evaluation_matches_oracle(lib, crane, name, N, K, S):
    import hulls
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints(name)
    s = _setup(lib, crane, name, N, K, S)
    try:
        xi = workloads.random_candidates(q0, qd, K, N, seed=4)
        g = s.evaluate(xi, q0, qd)
        J, Jc, pen = hulls.evaluate_hulls(s.problem, xi.astype(np.float64), q0, qd)
        np.testing.assert_allclose(g["pen"], pen, rtol=0, atol=TOL)
        flags = unpack_flags(g["words"], s.n_s)
        band = pen > 1e-4
        np.testing.assert_array_equal(flags[band], True)
        assert np.all(g["pen"][~flags] == 0.0)
        n_near = (pen > 0).sum(axis=1) + (g["pen"] > 0).sum(axis=1)
        assert np.all(np.abs(g["J"] - J) <= 1e-4 * np.abs(J) + 100.0 * TOL * n_near + 1e-9)
        assert band.sum() > 10
    finally:
        s.close()


def test_plan_with_hulls(lib, crane):
    """A plan on the hull model ends collision-free under that model (checked by the
    oracle), in the 20-tree stand."""
    import hulls
    q0, qd = endpoints("single_small")
    s = _setup(lib, crane, "single_small", 256, 8, 32)
    try:
        lib.cp_set_endpoints(s.h, q0, qd)
        ctrl, st = lib.cp_plan(s.h, 50, K=8)
        mu = ctrl[4:-4]
        J, Jc, pen = hulls.evaluate_hulls(s.problem, mu[None], q0, qd)
        n_near = int((pen > 0).sum()) + int(st["n_flagged"])
        assert abs(st["J"] - J[0]) <= 1e-4 * abs(J[0]) + 100.0 * TOL * n_near + 1e-9
        if pen.max() > 1e-4:
            assert st["flag"] == 1
        if st["flag"] == 0:
            assert pen.max() < TOL
    finally:
        s.close()

"""GPU parity of the CMA-ES update rule (the evolution strategy Algorithm 1 is modelled on)
against the oracle's update_cmaes: one update from an identical state (mean, covariance,
step size, both paths, iteration) on identical candidates and costs, with h_sigma on
either side of its threshold; free-space plans against the oracle's plan with the same
rule; and checkpoint / resume of the extended state.

Tolerances: the update is FP64 on both sides from the same float32 candidates. The mean
and the covariance carry a few FP64 roundings per elite (1e-12 relative); the step-size
path goes through the GPU's own FP64 Cholesky factor and a forward substitution
(1e-10 absolute on unit-scale paths for the well-conditioned covariances used here).
"""
import numpy as np
import pytest

from helpers import Setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


def _state(D, seed, p_sigma_scale):
    g = np.random.default_rng(seed)
    A = g.normal(size=(D, D))
    C = 0.05 * (A @ A.T / D + 0.3 * np.eye(D))
    mu = g.normal(size=D)
    return mu, C, 0.6, p_sigma_scale * g.normal(size=D), 0.3 * g.normal(size=D)


@pytest.mark.parametrize("N,K,t,ps,nu", [(256, 8, 5, 0.5, 0), (300, 4, 0, 0.2, 150), (4096, 16, 40, 6.0, 0),
                                         (9000, 8, 3, 1.0, 0)])
def test_update_matches_oracle(lib, crane, N, K, t, ps, nu):
    """ps = 6 puts |p_sigma| far above the h_sigma threshold (the rank-one path stalls);
    9000 candidates take the radix ranking."""
    import torch
    from paper_2503_14160_gb300 import workloads
    s = Setup(crane, workloads.empty_scene(), N=N, K=K, S=2, n_elites=nu, update_rule=1)
    try:
        D = 4 * K
        mu, C, sigma, p_sigma, p_c = _state(D, seed=N + K, p_sigma_scale=ps)
        lib.cp_set_endpoints(s.h, np.zeros(4), np.ones(4))
        state = np.concatenate([[sigma], p_sigma, p_c])
        lib.cp_set_cma_state(s.h, torch.from_numpy(state).cuda())
        lib.cp_set_distribution(s.h, torch.from_numpy(mu).cuda(), torch.from_numpy(C).cuda(), t)
        g = np.random.default_rng(N)
        Lc = np.linalg.cholesky(C)
        xi = (mu[None, :] + sigma * g.normal(size=(N, D)) @ Lc.T).astype(np.float32).reshape(N, K, 4)
        # neutral selection keeps |p_sigma| near its expectation (h_sigma = 1); costs that
        # pull the mean far in one direction push it over the threshold
        J = (g.random(N) if ps < 3.0 else
             np.sum((xi.reshape(N, D).astype(np.float64) - 0.3) ** 2, axis=1))
        lib.cp_update(s.h, torch.from_numpy(J).cuda(), torch.from_numpy(xi).cuda())
        mu_g = torch.zeros(D, dtype=torch.float64, device="cuda")
        C_g = torch.zeros(D, D, dtype=torch.float64, device="cuda")
        st_g = torch.zeros(1 + 2 * D, dtype=torch.float64, device="cuda")
        L_g = torch.zeros(D, D, dtype=torch.float64, device="cuda")
        lib.cp_get_distribution(s.h, mu_g, C_g)
        lib.cp_get_cma_state(s.h, st_g)
        lib.cp_get_factor(s.h, L_g)
        lib.cp_synchronize(s.h)
        st_o = s.oracle.CMAState(mu, C, sigma, p_sigma, p_c, t)
        new = s.oracle.update_cmaes(st_o, xi.astype(np.float64), J, s.nu)
        k = s.oracle.cma_constants(D, s.oracle.log_rank_weights(s.nu))
        h = np.linalg.norm(new.p_sigma) / np.sqrt(1 - (1 - k.c_sigma) ** (2 * (t + 1))) \
            < (1.4 + 2 / (D + 1)) * k.chi_n
        assert h == (ps < 3.0)
        sg = st_g.cpu().numpy()
        np.testing.assert_allclose(mu_g.cpu().numpy(), new.mu, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(sg[1:1 + D], new.p_sigma, rtol=0, atol=1e-10)
        np.testing.assert_allclose(sg[1 + D:], new.p_c, rtol=0, atol=1e-10)
        assert sg[0] == pytest.approx(new.sigma, rel=1e-11)
        Cg = C_g.cpu().numpy()
        np.testing.assert_allclose(Cg, new.C, rtol=1e-10, atol=1e-13 * np.abs(new.C).max())
        np.testing.assert_array_equal(Cg, Cg.T)
        np.testing.assert_allclose(L_g.cpu().numpy(), np.linalg.cholesky(sg[0] ** 2 * Cg), rtol=1e-11,
                                   atol=1e-14)
    finally:
        s.close()


def test_plan_free_space_matches_oracle(lib, crane):
    """No obstacles: the CMA-ES rule converges to the straight segment, an order of
    magnitude closer than the fixed-sigma rule's 1.5e-4 (the FP64 oracle reaches 1e-11; the
    GPU's FP32 costs stop the ranking near 1e-6), with the oracle's J_p, and the step size
    shrinks with the search."""
    from paper_2503_14160_gb300 import workloads
    q0 = np.array([2.0, 0.1, -2.0, 0.3])
    qd = np.array([-1.5, 1.0, -0.5, 2.2])
    s = Setup(crane, workloads.empty_scene(), N=128, K=6, S=16, seed=3, update_rule=1)
    try:
        import torch
        lib.cp_set_endpoints(s.h, q0, qd)
        ctrl, st = lib.cp_plan(s.h, 150, K=6)
        res = s.oracle.plan(s.problem, s.sp, q0, qd, 150, rule="cmaes")
        straight = np.linalg.norm(qd - q0)
        assert st["length"] == pytest.approx(straight, rel=1e-5)
        assert res.final.length[0] == pytest.approx(straight, rel=1e-7)
        assert st["Jp"] == pytest.approx(res.final.Jp[0], rel=1e-5)
        state = torch.zeros(1 + 2 * 24, dtype=torch.float64, device="cuda")
        lib.cp_get_cma_state(s.h, state)
        lib.cp_synchronize(s.h)
        assert state[0].item() < 1e-2   # from 1: the step size has shrunk with the search
    finally:
        s.close()


def test_resume_with_cma_state(lib, crane):
    """(mu, C, t) with the CMA state restored repeat the remaining iterations bit for bit."""
    import torch
    from paper_2503_14160_gb300 import workloads
    from helpers import endpoints
    q0, qd = endpoints("single_small")
    s = Setup(crane, workloads.make_scene(workloads.WORKLOADS["single_small"]), N=256, K=8, S=32,
              seed=5, update_rule=1)
    try:
        D = 32
        lib.cp_set_endpoints(s.h, q0, qd)
        a, _ = lib.cp_plan(s.h, 20, K=8)
        lib.cp_set_endpoints(s.h, q0, qd)
        lib.cp_plan(s.h, 10, K=8)
        mu = torch.zeros(D, dtype=torch.float64, device="cuda")
        C = torch.zeros(D, D, dtype=torch.float64, device="cuda")
        state = torch.zeros(1 + 2 * D, dtype=torch.float64, device="cuda")
        lib.cp_get_distribution(s.h, mu, C)
        lib.cp_get_cma_state(s.h, state)
        lib.cp_synchronize(s.h)
        lib.cp_set_endpoints(s.h, q0, qd)
        lib.cp_set_cma_state(s.h, state)
        lib.cp_set_distribution(s.h, mu, C, 10)
        b, st = lib.cp_plan(s.h, 10, K=8)
        np.testing.assert_array_equal(a, b)
        assert st["iteration"] == 20
    finally:
        s.close()


def test_paper_rule_state_is_fixed_sigma(lib, crane):
    import torch
    from paper_2503_14160_gb300 import workloads
    s = Setup(crane, workloads.empty_scene(), N=64, K=2, S=2, sigma=0.7)
    try:
        lib.cp_set_endpoints(s.h, np.zeros(4), np.ones(4))
        lib.cp_plan(s.h, 3, K=2)
        state = torch.ones(1 + 16, dtype=torch.float64, device="cuda")
        lib.cp_get_cma_state(s.h, state)
        lib.cp_synchronize(s.h)
        v = state.cpu().numpy()
        assert v[0] == 0.7 and np.all(v[1:] == 0.0)
    finally:
        s.close()

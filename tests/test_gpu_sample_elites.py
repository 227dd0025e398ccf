"""GPU parity of the factor-free sampler (step (1) from the last update's elites) with the
oracle's sample_elites, on identical updates: the mean to FP64 rounding, the samples within
the error bound of the tensor-core product, the covariance formed on request equal to the
paper's update, plans against the oracle's plan with the same sampler, and determinism.

Bound per sample coordinate (u = 2^-24). Y is formed in FP32 against the mean as an FP32
pair, within 4 ulp (8 u) of its FP64 value. The product sum_j g_ij Y_jd runs on the tensor
cores as G_hi Y_hi + G_hi Y_lo + G_lo Y_hi with G = G_hi + G_lo (+ a rest below 2^-22 |G|)
and the same split of Y: each product is within (12 + 8) u of g_ij Y_jd. The 3 nu products
are accumulated in FP32 (at most one ulp, 2 u, per addition even when the hardware
truncates) and the slices added in FP32, so the sum is within
(20 + 6 nu + slices + 16) u sum_j |g_ij||Y_jd| in the worst case; the float Box-Muller
normals add a few ulp each, the result's rounding u |xi|. Typical errors are far smaller:
independent rounding errors grow like sqrt(3 nu), and the RMS over all coordinates must
stay within (20 + 2 sqrt(3 nu)) u of the same scale.
"""
import numpy as np
import pytest

from helpers import Setup, endpoints

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


@pytest.mark.parametrize("N,K,nu,it", [(300, 4, 150, 3), (77, 1, 0, 0), (4096, 16, 0, 12), (256, 32, 0, 1),
                                       (9000, 8, 0, 7)])
def test_sample_matches_oracle(lib, crane, N, K, nu, it):
    """K = 1 (D = 4), K = 32 (two coordinate tiles), nu not a multiple of the 32-elite
    chunk (38), and the radix rank path (9000 candidates)."""
    import torch
    from paper_2503_14160_gb300 import workloads
    s = Setup(crane, workloads.empty_scene(), N=N, K=K, S=2, n_elites=nu, seed=21, sigma=0.8, eps=1e-6)
    s.planner.close()
    params = lib.make_params(N, K, 2, n_elites=nu, seed=21, sigma=0.8, eps=1e-6, query=2,
                             sampler=lib.CP_SAMPLE_ELITES)
    s.planner = lib.Planner(crane, workloads.empty_scene(), params)
    try:
        D = 4 * K
        g = np.random.default_rng(N + K)
        xi = (g.normal(size=(N, K, 4)) * 0.3 + 1.0).astype(np.float32)
        J = g.random(N)
        lib.cp_set_endpoints(s.h, np.zeros(4), np.ones(4))
        lib.cp_update(s.h, torch.from_numpy(J).cuda(), torch.from_numpy(xi).cuda())
        mu = torch.zeros(D, dtype=torch.float64, device="cuda")
        lib.cp_get_distribution(s.h, mu, None)
        out = torch.zeros(N, K, 4, device="cuda")
        lib.cp_sample(s.h, it, out)
        lib.cp_synchronize(s.h)
        nu_ = s.planner.nu
        mu_o, C_o = s.oracle.update(xi.astype(np.float64), J, nu_, 1e-6)
        np.testing.assert_allclose(mu.cpu().numpy(), mu_o, rtol=1e-12, atol=1e-14)
        order = s.oracle.rank(J)
        X = xi.reshape(N, D).astype(np.float64)[order[:nu_]]
        w = s.oracle.log_rank_weights(nu_)
        want = s.oracle.sample_elites(mu_o, X, w, 0.8, 1e-6, 21, it, 2, N, K).reshape(N, D)
        got = out.cpu().numpy().reshape(N, D).astype(np.float64)
        z = s.oracle.normals(21, it, 2, N, (nu_ + D + 3) // 4)
        Y = np.sqrt(w)[:, None] * (X - mu_o[None, :]) * 0.8
        scale = np.abs(z[:, :nu_]) @ np.abs(Y)
        bound = (EPS32 * np.abs(want) + (20 + 6 * nu_ + 32 + 16) * EPS32 * scale
                 + 8 * EPS32 * 0.8e-3 * np.abs(z[:, nu_:nu_ + D]) + 1e-30)
        err = np.abs(got - want)
        assert np.all(err <= bound), np.max(err / bound)
        rms = np.sqrt(np.mean((err / (scale + 1e-30)) ** 2))
        assert rms <= (20 + 2 * np.sqrt(3 * nu_)) * EPS32, rms / EPS32
    finally:
        s.close()


def test_covariance_on_request_is_the_update(lib, crane):
    """cp_get_distribution forms C from the current elites (the paper's update) without
    touching the mean the sampler uses; cp_get_factor returns its Cholesky factor."""
    import torch
    from paper_2503_14160_gb300 import workloads
    N, K = 500, 6
    D = 4 * K
    params = lib.make_params(N, K, 2, eps=1e-8, sampler=lib.CP_SAMPLE_ELITES)
    pl = lib.Planner(crane, workloads.empty_scene(), params)
    try:
        import oracle
        g = np.random.default_rng(3)
        xi = (g.normal(size=(N, K, 4)) * 0.2).astype(np.float32)
        J = g.random(N)
        lib.cp_set_endpoints(pl.handle, np.zeros(4), np.ones(4))
        lib.cp_update(pl.handle, torch.from_numpy(J).cuda(), torch.from_numpy(xi).cuda())
        mu0 = torch.zeros(D, dtype=torch.float64, device="cuda")
        lib.cp_get_distribution(pl.handle, mu0, None)
        mu1 = torch.zeros(D, dtype=torch.float64, device="cuda")
        C = torch.zeros(D, D, dtype=torch.float64, device="cuda")
        Lg = torch.zeros(D, D, dtype=torch.float64, device="cuda")
        lib.cp_get_distribution(pl.handle, mu1, C)
        lib.cp_get_factor(pl.handle, Lg)
        lib.cp_synchronize(pl.handle)
        np.testing.assert_array_equal(mu0.cpu().numpy(), mu1.cpu().numpy())
        mu_o, C_o = oracle.update(xi.astype(np.float64), J, N // 2, 1e-8)
        Cg = C.cpu().numpy()
        np.testing.assert_allclose(Cg, C_o, rtol=1e-11, atol=1e-14 * np.abs(C_o).max())
        np.testing.assert_allclose(Lg.cpu().numpy(), np.linalg.cholesky(Cg), rtol=1e-11, atol=1e-14)
    finally:
        pl.close()


def test_plan_free_space_matches_oracle(lib, crane):
    from paper_2503_14160_gb300 import workloads
    q0 = np.array([2.0, 0.1, -2.0, 0.3])
    qd = np.array([-1.5, 1.0, -0.5, 2.2])
    s = Setup(crane, workloads.empty_scene(), N=128, K=6, S=16, seed=3)
    s.planner.close()
    s.planner = lib.Planner(crane, workloads.empty_scene(),
                            lib.make_params(128, 6, 16, seed=3, sampler=lib.CP_SAMPLE_ELITES))
    try:
        lib.cp_set_endpoints(s.h, q0, qd)
        ctrl, st = lib.cp_plan(s.h, 150, K=6)
        res = s.oracle.plan(s.problem, s.sp, q0, qd, 150, sampler="elites")
        assert st["length"] == pytest.approx(np.linalg.norm(qd - q0), rel=1e-3)
        assert st["length"] == pytest.approx(res.final.length[0], rel=1e-3)
        assert st["Jp"] == pytest.approx(res.final.Jp[0], rel=1e-3)
        assert st["flag"] == 0
    finally:
        s.close()


def test_plans_repeat_and_graphs_agree(lib, crane):
    """Same seed, same plan bit for bit; on a stream of the caller's (recorded graph) as on
    the default stream."""
    import torch
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("single_small")
    scene = workloads.make_scene(workloads.WORKLOADS["single_small"])
    params = lib.make_params(256, 8, 32, seed=5, sampler=lib.CP_SAMPLE_ELITES)
    a = lib.Planner(crane, scene, params)
    b = lib.Planner(crane, scene, params, stream=torch.cuda.Stream())
    try:
        res = []
        for pl in (a, a, b, b):
            lib.cp_set_endpoints(pl.handle, q0, qd)
            res.append(lib.cp_plan(pl.handle, 15, K=8)[0])
        for r in res[1:]:
            np.testing.assert_array_equal(res[0], r)
    finally:
        a.close()
        b.close()


def test_needs_the_paper_rule(lib, crane):
    from paper_2503_14160_gb300 import workloads
    with pytest.raises(Exception):
        lib.Planner(crane, workloads.empty_scene(),
                    lib.make_params(64, 2, 2, update_rule=lib.CP_UPDATE_CMAES, sampler=lib.CP_SAMPLE_ELITES))


def test_unaligned_candidates_are_rejected(lib, crane):
    """Candidate arrays move one control point (16 bytes) at a time: a pointer off by one
    float is refused on the host, before any launch."""
    import torch
    from paper_2503_14160_gb300 import workloads
    pl = lib.Planner(crane, workloads.empty_scene(), lib.make_params(64, 2, 2, sampler=lib.CP_SAMPLE_ELITES))
    try:
        lib.cp_set_endpoints(pl.handle, np.zeros(4), np.ones(4))
        buf = torch.zeros(64 * 8 + 1, device="cuda")
        J = torch.zeros(64, dtype=torch.float64, device="cuda")
        off = buf.data_ptr() + 4
        for call in (lambda: lib.cp_sample(pl.handle, 0, off), lambda: lib.cp_evaluate(pl.handle, off, 64, J),
                     lambda: lib.cp_update(pl.handle, J, off)):
            with pytest.raises(lib.CranePlanError, match="aligned"):
                call()
        lib.cp_sample(pl.handle, 0, buf[:-1])   # the aligned start is fine
        lib.cp_synchronize(pl.handle)
    finally:
        pl.close()


def test_operand_wait_runs_out_and_is_reported(lib, crane):
    """With the operand copy withheld (test hook 2) the MMA warp's bounded wait for it runs
    out: the launch still finishes and releases its tensor memory, CP_ERR_TIMEOUT is
    reported at the next synchronisation, and the device keeps working."""
    import time
    import torch
    from paper_2503_14160_gb300 import workloads
    N, K = 64, 2
    bad = lib.Planner(crane, workloads.empty_scene(),
                      lib.make_params(N, K, 2, sampler=lib.CP_SAMPLE_ELITES, debug_withhold_staging=2))
    try:
        g = np.random.default_rng(5)
        xi = torch.from_numpy((g.normal(size=(N, K, 4)) * 0.3).astype(np.float32)).cuda()
        J = torch.from_numpy(g.random(N)).cuda()
        lib.cp_set_endpoints(bad.handle, np.zeros(4), np.ones(4))
        lib.cp_update(bad.handle, J, xi)
        lib.cp_synchronize(bad.handle)
        out = torch.zeros(N, K, 4, device="cuda")
        t0 = time.perf_counter()
        lib.cp_sample(bad.handle, 1, out)
        with pytest.raises(lib.CranePlanError) as e:
            lib.cp_synchronize(bad.handle)
        assert e.value.status == -3
        assert time.perf_counter() - t0 < 30.0
        lib.cp_synchronize(bad.handle)          # the report is cleared once read
    finally:
        bad.close()
    s = Setup(crane, workloads.empty_scene(), N=N, K=K, S=2, seed=21, sigma=0.8, eps=1e-6)
    s.planner.close()
    s.planner = lib.Planner(crane, workloads.empty_scene(),
                            lib.make_params(N, K, 2, seed=21, sigma=0.8, eps=1e-6, sampler=lib.CP_SAMPLE_ELITES))
    try:                                         # the device keeps working: a clean draw
        lib.cp_set_endpoints(s.h, np.zeros(4), np.ones(4))
        g = np.random.default_rng(6)
        xi = torch.from_numpy((g.normal(size=(N, K, 4)) * 0.3).astype(np.float32)).cuda()
        lib.cp_update(s.h, torch.from_numpy(g.random(N)).cuda(), xi)
        out = torch.zeros(N, K, 4, device="cuda")
        lib.cp_sample(s.h, 1, out)
        lib.cp_synchronize(s.h)
        assert torch.isfinite(out).all()
    finally:
        s.close()

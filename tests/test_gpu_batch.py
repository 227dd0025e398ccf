"""The batched serving form (Algorithm 1 for many queries; arXiv 2503.14160, Sec. 4.1 and the
many-query setting of Sec. 5.1): every stage of an iteration is one launch for all queries,
the evaluation a persistent launch over a device queue of tiles.

  - Each query's plan equals, bit for bit, the plan of its planner alone (the batched kernels
    share the single-query kernels' per-item, per-candidate and per-entry arithmetic, and the
    segmented ranking gives the plain ranking's order), for every launch shape.
  - One iteration of several uneven queries against the oracle: the draw, every candidate's
    cost, the ranking, the updated mean and covariance, and the mean path's cost.
"""
import numpy as np
import pytest

from helpers import D_TOL, cost_tolerance, factor_sample_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


def _queries(crane, sizes, S):
    import oracle
    from paper_2503_14160_gb300 import craneplan as cp, workloads
    scenes, params, q0s, qds, raw = [], [], [], [], []
    for q, (N, K, M, cell) in enumerate(sizes):
        bq = workloads.BatchQuery(N, K, M, float(np.sqrt(4.0 + M / (1.66 * np.pi))))
        sc = workloads.batch_scene(bq, seed=0, q=q)
        pb = oracle.Problem(crane, sc, oracle.CostParams(K=K, S=S))
        q0, qd, ok, _ = workloads.select_endpoints(crane, lambda x: oracle.signed_distance(pb, x),
                                                   seed=0, batch=4096, query=q)
        raw.append(sc)
        scenes.append(cp.HostScene.from_scene(sc))
        params.append(cp.make_params(N, K, S, seed=q, query=q, grid_cell=cell))
        q0s.append(q0)
        qds.append(qd)
    return scenes, params, q0s, qds, raw


# (N, K, cylinders, ring width of the polar index): uneven sizes, an empty scene, a ragged N,
# and one population above 8192 (ranked by the radix sort when planned alone)
SIZES = [(64, 2, 5, 0.5), (200, 5, 40, 0.75), (33, 8, 60, 0.5), (128, 3, 0, 1.0), (9000, 2, 30, 1.0),
         (96, 4, 20, 1.0)]


def test_batch_matches_plain_plans(lib):
    from paper_2503_14160_gb300 import workloads
    cp = lib
    crane = workloads.forestry_crane()
    model = cp.make_model(crane)
    S, T = 8, 6
    scenes, params, q0s, qds, _ = _queries(crane, SIZES, S)
    Ks = [s[1] for s in SIZES]
    nq = len(SIZES)
    b = cp.cp_batch_init(model, scenes, params, q0s, qds, T)
    try:
        info = cp.cp_batch_get_info(b)
        assert info["eval_launches"] == T + 1
        assert info["candidates"] == sum(s[0] for s in SIZES)
        # per iteration: sample, evaluation, costs, ranking (init + 9 passes x 3), gather,
        # moments (deviations, partials, first moments, combine), factor
        assert info["kernel_nodes"] == 2 + T * (1 + 1 + 1 + 1 + 9 * 3 + 1 + 4 + 1) + 4
        res = cp.cp_batch_run(b, nq, K=Ks)
        # every launch shape gives the same bits
        for shape in [(128, 1, 1), (512, 0, 8), (256, 2, 64)]:
            cp.cp_batch_set_shape(b, *shape)
            again = cp.cp_batch_run(b, nq, K=Ks)
            for q in range(nq):
                np.testing.assert_array_equal(again[q][0], res[q][0])
                assert again[q][1]["J"] == res[q][1]["J"]
        for q in range(nq):
            p = cp.cp_batch_planner(b, q)
            cp.cp_set_endpoints(p, q0s[q], qds[q])
            ctrl, st = cp.cp_plan(p, T, K=Ks[q])
            np.testing.assert_array_equal(res[q][0], ctrl)
            assert res[q][1]["J"] == st["J"] and res[q][1]["length"] == st["length"]
            assert res[q][1]["best_J"] == st["best_J"]
            assert res[q][1]["n_flagged"] == st["n_flagged"]
        # new end points for query 1 (swap start and goal)
        cp.cp_batch_set_endpoints(b, 1, qds[1], q0s[1])
        swapped = cp.cp_batch_run(b, nq, K=Ks)
        p = cp.cp_batch_planner(b, 1)
        cp.cp_set_endpoints(p, qds[1], q0s[1])
        ctrl, st = cp.cp_plan(p, T, K=Ks[1])
        np.testing.assert_array_equal(swapped[1][0], ctrl)
        np.testing.assert_array_equal(swapped[0][0], res[0][0])
        np.testing.assert_array_equal(swapped[1][0][:4], np.tile(qds[1], (4, 1)))
    finally:
        cp.cp_batch_destroy(b)


def test_batch_one_iteration_against_oracle(lib):
    """Queries of uneven N, K and obstacle count, one iteration: step (1) against the
    oracle's draw from the same Philox counters, step (2) on every candidate against the
    oracle's FP64 cost of the same FP32 candidate,
    step (3) the ranking of the GPU's costs exactly (index work), steps (4)-(6) the updated
    mean and covariance from those elites, and the mean path's cost and length."""
    import torch
    import oracle
    from paper_2503_14160_gb300 import workloads
    cp = lib
    crane = workloads.forestry_crane()
    model = cp.make_model(crane)
    S = 16
    sizes = [(300, 3, 120, 0.5), (77, 6, 400, 0.75), (512, 2, 50, 1.0), (129, 5, 900, 0.5)]
    scenes, params, q0s, qds, raw = _queries(crane, sizes, S)
    Ks = [s[1] for s in sizes]
    b = cp.cp_batch_init(model, scenes, params, q0s, qds, 1)
    try:
        res = cp.cp_batch_run(b, len(sizes), K=Ks)
        for q, (N, K, M, _) in enumerate(sizes):
            D = 4 * K
            p = cp.cp_batch_planner(b, q)
            xi = torch.zeros(N, K, 4, device="cuda")
            J = torch.zeros(N, dtype=torch.float64, device="cuda")
            cp.cp_get_population(p, xi, J)
            mu_g = torch.zeros(D, dtype=torch.float64, device="cuda")
            C_g = torch.zeros(D, D, dtype=torch.float64, device="cuda")
            cp.cp_get_distribution(p, mu_g, C_g)
            sp = oracle.SearchParams(N=N, K=K, S=S, seed=q)
            nu = N // 2
            el = torch.zeros(nu, dtype=torch.int32, device="cuda")
            cp.cp_get_elites(p, el)
            torch.cuda.synchronize()
            X = xi.cpu().numpy().reshape(N, D).astype(np.float64)
            J_g = J.cpu().numpy()
            # step (1)
            mu0, C0 = oracle.init_distribution(q0s[q], qds[q], K, crane.q_min, crane.q_max)
            L0 = oracle.factor(C0, sp.sigma)
            want = oracle.sample(mu0, L0, sp.seed, 0, q, N, K).reshape(N, D)
            bound = factor_sample_bound(want, oracle.normals(sp.seed, 0, q, N, K), L0)
            assert np.all(np.abs(X - want) <= bound), q
            # step (2)
            pb = oracle.Problem(crane, raw[q], oracle.CostParams(K=K, S=S))
            o = oracle.evaluate(pb, X.reshape(N, K, 4), q0s[q], qds[q], with_distances=True)
            d = o.d[:, 1:]
            n_near = (d < D_TOL).sum(axis=1)
            tol = cost_tolerance(o.J, n_near)
            assert np.all(np.abs(J_g - o.J) <= tol), (q, np.max(np.abs(J_g - o.J) - tol))
            # step (3): the ranking of the GPU's costs by (J, index)
            np.testing.assert_array_equal(el.cpu().numpy(), oracle.rank(J_g)[:nu])
            # steps (4)-(6) from those elites
            mu_o, C_o = oracle.update(X, J_g, nu, sp.eps)
            np.testing.assert_allclose(mu_g.cpu().numpy(), mu_o, rtol=1e-12, atol=1e-13)
            np.testing.assert_allclose(C_g.cpu().numpy(), C_o, rtol=1e-11, atol=1e-13 * np.abs(C_o).max())
            # the mean path (the FP32 copy of the updated mean) against the oracle
            mean32 = mu_g.cpu().numpy().astype(np.float32).astype(np.float64).reshape(1, K, 4)
            om = oracle.evaluate(pb, mean32, q0s[q], qds[q], with_distances=True)
            n_near_m = (om.d[:, 1:] < D_TOL).sum(axis=1)
            st = res[q][1]
            assert abs(st["J"] - om.J[0]) <= cost_tolerance(om.J, n_near_m)[0]
            assert abs(st["length"] - om.length[0]) <= 2e-5 * om.length[0]
            assert st["best_J"] == J_g[oracle.rank(J_g)[0]]
            np.testing.assert_array_equal(res[q][0][4:K + 4], mu_g.cpu().numpy().reshape(K, 4))
    finally:
        cp.cp_batch_destroy(b)


def test_batch_rejects_bad_query(lib):
    from paper_2503_14160_gb300 import workloads
    cp = lib
    model = cp.make_model(workloads.forestry_crane())
    sc = cp.HostScene.from_scene(workloads.empty_scene())
    good = cp.make_params(16, 2, 4, grid_cell=0.5)
    bad = cp.make_params(16, 40, 4, grid_cell=0.5)
    with pytest.raises(cp.CranePlanError) as e:
        cp.cp_batch_init(model, [sc, sc], [good, bad], [np.zeros(4)] * 2, [np.ones(4)] * 2, 3)
    assert "query 1" in str(e.value)
    broad = cp.make_params(16, 2, 4)
    with pytest.raises(cp.CranePlanError) as e:
        cp.cp_batch_init(model, [sc, sc], [broad, good], [np.zeros(4)] * 2, [np.ones(4)] * 2, 3)
    assert "query 0" in str(e.value) and "polar" in str(e.value)
    elites = cp.make_params(16, 2, 4, grid_cell=0.5, sampler=cp.CP_SAMPLE_ELITES)
    with pytest.raises(cp.CranePlanError):
        cp.cp_batch_init(model, [sc], [elites], [np.zeros(4)], [np.ones(4)], 3)
    b = cp.cp_batch_init(model, [sc], [good], [np.zeros(4)], [np.ones(4)], 2)
    try:
        for shape in [(100, 0, 1), (256, -1, 1), (256, 0, 0), (256, 0, 65)]:
            with pytest.raises(cp.CranePlanError):
                cp.cp_batch_set_shape(b, *shape)
        cp.cp_batch_run(b, 1)   # the old shape still runs
    finally:
        cp.cp_batch_destroy(b)

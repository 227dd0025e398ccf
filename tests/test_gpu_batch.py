"""The batched serving form: uneven queries recorded into one CUDA graph give, query by
query, the same plan bit for bit as planning that query alone (the graph changes only the
scheduling, not the arithmetic); a replay repeats it; new end points take effect."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_batch_matches_plain_plans():
    import oracle
    from paper_2503_14160_gb300 import build, craneplan as cp, workloads
    build.build()
    cp.load()
    crane = workloads.forestry_crane()
    model = cp.make_model(crane)
    sizes = [(64, 2, 5, 0.0), (200, 5, 40, 0.0), (33, 8, 60, 0.5), (128, 3, 0, 0.0), (96, 4, 20, 1.0)]
    S, T = 8, 6
    scenes, params, q0s, qds = [], [], [], []
    for q, (N, K, M, cell) in enumerate(sizes):
        bq = workloads.BatchQuery(N, K, M, float(np.sqrt(4.0 + M / (1.66 * np.pi))))
        sc = workloads.batch_scene(bq, seed=0, q=q)
        pb = oracle.Problem(crane, sc, oracle.CostParams(K=K, S=S))
        q0, qd, ok, _ = workloads.select_endpoints(crane, lambda x: oracle.signed_distance(pb, x),
                                                   seed=0, batch=4096, query=q)
        scenes.append(cp.HostScene.from_scene(sc))
        params.append(cp.make_params(N, K, S, seed=q, query=q, grid_cell=cell))
        q0s.append(q0)
        qds.append(qd)
    Ks = [s[1] for s in sizes]
    b = cp.cp_batch_init(model, scenes, params, q0s, qds, T)
    try:
        res = cp.cp_batch_run(b, len(sizes), K=Ks)
        for q in range(len(sizes)):
            p = cp.cp_batch_planner(b, q)
            cp.cp_set_endpoints(p, q0s[q], qds[q])
            ctrl, st = cp.cp_plan(p, T, K=Ks[q])
            np.testing.assert_array_equal(res[q][0], ctrl)
            assert res[q][1]["J"] == st["J"] and res[q][1]["length"] == st["length"]
            assert res[q][1]["best_J"] == st["best_J"]
        again = cp.cp_batch_run(b, len(sizes), K=Ks)
        for q in range(len(sizes)):
            np.testing.assert_array_equal(again[q][0], res[q][0])
        # new end points for query 1 (swap start and goal)
        cp.cp_batch_set_endpoints(b, 1, qds[1], q0s[1])
        swapped = cp.cp_batch_run(b, len(sizes), K=Ks)
        p = cp.cp_batch_planner(b, 1)
        cp.cp_set_endpoints(p, qds[1], q0s[1])
        ctrl, st = cp.cp_plan(p, T, K=Ks[1])
        np.testing.assert_array_equal(swapped[1][0], ctrl)
        np.testing.assert_array_equal(swapped[0][0], res[0][0])
        np.testing.assert_array_equal(swapped[1][0][:4], np.tile(qds[1], (4, 1)))
    finally:
        cp.cp_batch_destroy(b)


def test_batch_rejects_bad_query():
    from paper_2503_14160_gb300 import build, craneplan as cp, workloads
    build.build()
    cp.load()
    model = cp.make_model(workloads.forestry_crane())
    sc = cp.HostScene.from_scene(workloads.empty_scene())
    good = cp.make_params(16, 2, 4)
    bad = cp.make_params(16, 40, 4)
    with pytest.raises(cp.CranePlanError) as e:
        cp.cp_batch_init(model, [sc, sc], [good, bad], [np.zeros(4)] * 2, [np.ones(4)] * 2, 3)
    assert "query 1" in str(e.value)

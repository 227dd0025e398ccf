"""GPU parity of Algorithm 1 step (2) (Eq. path opt) and of d(q) (Sec. 3.1): the CUDA
library against the FP64 oracle on identical seeded float32 candidates. Per checkpoint the
penalty max(0, -d) agrees within D_TOL and collision flags agree bit for bit wherever the
oracle's |d| exceeds 1e-4 m; per candidate J agrees within the tolerance of helpers.py."""
import numpy as np
import pytest

from helpers import D_TOL, FLAG_BAND, Setup, cost_tolerance, endpoints, unpack_flags

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


def _scene(name, n_cyl=None, n_box=None):
    from paper_2503_14160_gb300 import workloads
    sc = workloads.make_scene(workloads.WORKLOADS[name])
    cyl, box = sc.cylinders, sc.boxes
    if n_cyl is not None:   # nearest cylinders to the base (those the crane can reach)
        cyl = cyl[np.argsort(np.hypot(cyl[:, 0], cyl[:, 1]), kind="stable")[:n_cyl]]
    if n_box is not None:
        box = box[:n_box]
    return workloads.Scene(cyl, box)


def check_eval(setup, xi, q0, qd, idx=None):
    """Evaluate xi on the GPU; compare the candidates `idx` (all by default) with the oracle."""
    g = setup.evaluate(xi, q0, qd)
    idx = np.arange(xi.shape[0]) if idx is None else np.asarray(idx)
    o = setup.oracle.evaluate(setup.problem, xi[idx].astype(np.float64), q0, qd,
                              with_distances=True)
    d = o.d[:, 1:]                                   # checkpoints 1..n_s
    pen_o = np.maximum(0.0, -d)
    err = np.abs(g["pen"][idx] - pen_o)
    assert err.max() <= D_TOL, "per-checkpoint penalty off by %g m" % err.max()
    flags = unpack_flags(g["words"][idx], setup.n_s)
    band = np.abs(d) > FLAG_BAND
    mism = flags[band] != (d < 0)[band]
    assert not mism.any(), "%d flags differ outside the 1e-4 m band" % mism.sum()
    n_near = (d < D_TOL).sum(axis=1)
    tol = cost_tolerance(o.J, n_near, setup.problem.cost.w_c, setup.problem.cost.lambda_c)
    dJ = np.abs(g["J"][idx] - o.J)
    assert np.all(dJ <= tol), "J off: worst %g (tol %g)" % (dJ.max(), tol[np.argmax(dJ - tol)])
    t = g["terms"][idx]
    np.testing.assert_allclose(t[:, 0], o.Jp, rtol=2e-5, atol=1e-12)
    np.testing.assert_allclose(t[:, 3], o.length, rtol=2e-5, atol=1e-9)
    np.testing.assert_allclose(t[:, 2], o.Jl, rtol=1e-4, atol=1e-7 * setup.n_s)
    assert np.all(np.abs(t[:, 1] - o.Jc) <= setup.problem.cost.lambda_c * D_TOL * n_near + 1e-12)
    np.testing.assert_array_equal(t[:, 4], flags.sum(axis=1))
    np.testing.assert_array_equal(g["flag"][idx], flags.any(axis=1))
    clean = ~(np.abs(d) <= FLAG_BAND).any(axis=1)
    np.testing.assert_array_equal(g["flag"][idx][clean], o.flag[clean])
    return g, o


@pytest.mark.parametrize("K,S,n", [(8, 32, 256), (5, 7, 37), (1, 1, 2), (3, 33, 5)])
def test_evaluate_small_forest(lib, crane, K, S, n):
    """The 20-tree scene at the sizes of the plain query (K=8, S=32, N=256) and at ragged
    sizes (n_s not a multiple of 32, candidates not a multiple of the warps per CTA)."""
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("single_small")
    s = Setup(crane, _scene("single_small"), N=max(n, 2), K=K, S=S)
    try:
        xi = workloads.random_candidates(q0, qd, K, n, seed=K * 100 + S)
        g, o = check_eval(s, xi, q0, qd)
        d = o.d[:, 1:]
        if n >= 8:   # both sides of contact are exercised
            assert (d < 0).any() and (d > 0).any()
    finally:
        s.close()


def test_evaluate_boxes_and_dense_cylinders(lib, crane):
    """Cylinders and axis-aligned boxes together (the dense-forest obstacle types)."""
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("dense_forest")
    s = Setup(crane, _scene("dense_forest", n_cyl=300), N=64, K=4, S=16)
    try:
        xi = workloads.random_candidates(q0, qd, 4, 64, seed=5)
        check_eval(s, xi, q0, qd)
    finally:
        s.close()


def test_evaluate_empty_scene_and_n0(lib, crane):
    from paper_2503_14160_gb300 import workloads
    q0 = np.array([1.0, 0.5, -1.0, 0.5])
    qd = np.array([-1.0, 0.2, -2.0, 2.0])
    s = Setup(crane, workloads.empty_scene(), N=16, K=3, S=5)
    try:
        xi = workloads.random_candidates(q0, qd, 3, 16, seed=9)
        g, o = check_eval(s, xi, q0, qd)
        assert np.all(g["terms"][:, 1] == 0.0) and np.all(g["flag"] == 0)
        import torch
        J = torch.zeros(1, dtype=torch.float64, device="cuda")
        xi_t = torch.zeros(1, 3, 4, device="cuda")
        lib.cp_evaluate(s.h, xi_t, 0, J)           # n = 0 is a no-op
        with pytest.raises(lib.CranePlanError):
            lib.cp_evaluate(s.h, xi_t, 17, J)     # n > N
    finally:
        s.close()


def test_evaluate_straight_line_free_space(lib, crane):
    """Evenly spaced control points: length |qd - q0|, no penalties."""
    from paper_2503_14160_gb300 import workloads
    q0 = np.array([2.0, 0.1, -2.0, 0.3])
    qd = np.array([-1.5, 1.0, -0.5, 2.2])
    s = Setup(crane, workloads.empty_scene(), N=4, K=8, S=32)
    try:
        xi = workloads.straight_line_points(q0, qd, 8)[None].astype(np.float32)
        g = s.evaluate(xi, q0, qd)
        assert g["terms"][0, 3] == pytest.approx(np.linalg.norm(qd - q0), rel=1e-5)
        assert g["terms"][0, 1] == 0.0 and g["terms"][0, 2] == 0.0
    finally:
        s.close()


def test_evaluate_max_waypoints(lib, crane):
    """K = 32 (the largest) with 128 checkpoints per span: n_s = 4480."""
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("single_small")
    s = Setup(crane, _scene("single_small"), N=6, K=32, S=128)
    try:
        xi = workloads.random_candidates(q0, qd, 32, 6, seed=3)
        check_eval(s, xi, q0, qd)
    finally:
        s.close()


def test_evaluate_single_large_full_size(lib, crane):
    """The single large query at its full size (N=4096, K=16, S=64, 500 trees), evaluated
    on the GPU in one launch; the oracle checks 24 candidates spread over the population
    (including the first and last, so every warp position and the grid tail are covered)."""
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("single_large")
    s = Setup(crane, _scene("single_large"), N=4096, K=16, S=64)
    try:
        xi = workloads.random_candidates(q0, qd, 16, 4096, seed=21, spread=(0.3, 0.15, 0.2, 0.3))
        idx = np.unique(np.r_[0, 1, 31, 32, np.linspace(0, 4095, 20).astype(int), 4095])
        check_eval(s, xi, q0, qd, idx)
    finally:
        s.close()


@pytest.mark.parametrize("half,cell", [(0.0, 0.5), (5.0, 0.5), (0.0, 0.23)])
def test_evaluate_grid_dense_forest(lib, crane, half, cell):
    """The polar-index evaluation on the dense forest (5000 cylinders + 50 boxes) against the
    oracle's brute force: the default rings, closed rings only to 5 m (spheres beyond it
    query the open last ring that holds every farther obstacle) and an odd ring width."""
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("dense_forest")
    s = Setup(crane, workloads.make_scene(workloads.WORKLOADS["dense_forest"]), N=64, K=6,
              S=16, grid_cell=cell, grid_half_extent=half)
    try:
        xi = workloads.random_candidates(q0, qd, 6, 64, seed=17)
        g, o = check_eval(s, xi, q0, qd)
        assert (o.d[:, 1:] < 0).any() and (o.d[:, 1:] > 0).any()
    finally:
        s.close()


def test_evaluate_grid_dense_forest_full_size(lib, crane):
    """The dense forest at its full size (N=65536, K=32, S=128) in one launch; the oracle
    checks 8 candidates spread over the population."""
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("dense_forest")
    s = Setup(crane, workloads.make_scene(workloads.WORKLOADS["dense_forest"]), N=65536, K=32,
              S=128, grid_cell=0.5)
    try:
        xi = workloads.random_candidates(q0, qd, 32, 65536, seed=23, spread=(0.3, 0.15, 0.2, 0.3))
        idx = np.array([0, 31, 32, 20000, 40000, 65503, 65504, 65535])
        check_eval(s, xi, q0, qd, idx)
    finally:
        s.close()


@pytest.mark.parametrize("name,n_cyl,K,S,n,spread", [
    ("single_small", None, 8, 32, 256, (0.6, 0.3, 0.4, 0.5)),
    ("single_large", None, 16, 64, 512, (0.6, 0.3, 0.4, 0.5)),
    ("single_large", None, 5, 7, 45, (3.0, 1.0, 1.5, 2.0)),     # far outside the limits
    ("dense_forest", 300, 4, 16, 64, (0.6, 0.3, 0.4, 0.5)),     # cylinders and boxes
    ("dense_forest", None, 6, 16, 40, (0.6, 0.3, 0.4, 0.5)),    # 5000 cylinders, no grid
])
def test_broadphase_matches_exhaustive_bitwise(lib, crane, name, n_cyl, K, S, n, spread):
    """The broad phase and the polar index only drop obstacles that no sphere of the 32
    checkpoints can reach, and they take the same exact distances, so the default
    evaluation, the polar-index one (two ring widths) and the exhaustive one (every sphere
    against every obstacle) give the same penalties, flags, terms and costs bit for bit."""
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints(name)
    scene = _scene(name, n_cyl=n_cyl)
    xi = workloads.random_candidates(q0, qd, K, n, seed=K * 7 + n, spread=spread)
    out = []
    for exhaustive, cell in ((0, 0.0), (1, 0.0), (0, 0.5), (0, 1.7)):
        s = Setup(crane, scene, N=n, K=K, S=S, exhaustive=exhaustive, grid_cell=cell)
        try:
            out.append(s.evaluate(xi, q0, qd))
        finally:
            s.close()
    for other in out[1:]:
        for key in ("J", "flag", "terms", "words", "pen"):
            np.testing.assert_array_equal(out[0][key], other[key], err_msg=key)
    assert out[0]["flag"].any()


def test_evaluate_spheres_of_unequal_radius(lib, crane):
    """A model whose spheres differ in radius (the filter bound uses the largest); checked
    against the oracle."""
    import dataclasses
    from paper_2503_14160_gb300 import workloads
    spheres = tuple(dataclasses.replace(sp, radius=0.25 + 0.02 * (i % 3))
                    for i, sp in enumerate(crane.spheres))
    model = dataclasses.replace(crane, spheres=spheres)
    q0, qd = endpoints("single_small")
    s = Setup(model, _scene("single_small"), N=64, K=6, S=20)
    try:
        xi = workloads.random_candidates(q0, qd, 6, 64, seed=31)
        g, o = check_eval(s, xi, q0, qd)
        assert (o.d[:, 1:] < 0).any()
    finally:
        s.close()


def test_work_counters(lib, crane):
    """While timing is on the planner reports the evaluation work: units, and obstacle
    tests (every obstacle of every unit when exhaustive, the counted broad-phase survivors
    otherwise, a small fraction of them on the 500-tree scene)."""
    import torch
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("single_large")
    scene = _scene("single_large")
    n, K, S = 256, 16, 64
    xi = torch.from_numpy(workloads.random_candidates(q0, qd, K, n, seed=4)).cuda()
    J = torch.zeros(n, dtype=torch.float64, device="cuda")
    chunks = ((K + 3) * S + 31) // 32
    got = []
    for exhaustive in (1, 0):
        s = Setup(crane, scene, N=n, K=K, S=S, exhaustive=exhaustive)
        try:
            lib.cp_set_endpoints(s.h, q0, qd)
            lib.cp_set_timing(s.h, True)
            lib.cp_evaluate(s.h, xi, n, J)
            lib.cp_evaluate(s.h, xi, n, J)
            t = lib.cp_get_timing(s.h)
            lib.cp_set_timing(s.h, False)
        finally:
            s.close()
        assert t["eval_launches"] == 2 and t["eval_units"] == 2 * n * chunks
        assert t["eval_pair_tests"] == 32 * 12 * t["eval_obstacle_tests"]
        assert t["eval_box_tests"] == -1
        got.append(t["eval_obstacle_tests"])
    assert got[0] == 2 * n * chunks * scene.n_cyl
    assert 0 < got[1] < got[0] // 10
    # polar-index form: the obstacles listed for each checkpoint (a small fraction of the
    # scene) and those whose filter passed
    s = Setup(crane, scene, N=n, K=K, S=S, grid_cell=0.5)
    try:
        lib.cp_set_endpoints(s.h, q0, qd)
        lib.cp_set_timing(s.h, True)
        lib.cp_evaluate(s.h, xi, n, J)
        t = lib.cp_get_timing(s.h)
        lib.cp_set_timing(s.h, False)
    finally:
        s.close()
    n_s = (K + 3) * S
    assert t["eval_units"] == n * chunks
    assert 0 < t["eval_obstacle_tests"] <= t["eval_box_tests"] < n * n_s * scene.n_cyl // 20
    assert t["eval_pair_tests"] == 12 * t["eval_box_tests"]


def test_exhaustive_matches_oracle(lib, crane):
    """The exhaustive evaluation against the oracle directly (boxes and cylinders)."""
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("dense_forest")
    s = Setup(crane, _scene("dense_forest", n_cyl=200), N=48, K=5, S=12, exhaustive=1)
    try:
        check_eval(s, workloads.random_candidates(q0, qd, 5, 48, seed=8), q0, qd)
    finally:
        s.close()


def test_signed_distance(lib, crane):
    """d(q) for configurations inside and beyond the joint limits."""
    import torch
    from paper_2503_14160_gb300 import workloads
    s = Setup(crane, _scene("dense_forest", n_cyl=400, n_box=50), N=4, K=2, S=2)
    try:
        g = workloads.rng(0, workloads.STREAM_TEST, 1)
        q = workloads.uniform_configurations(crane, g, 4096)
        q[:256] *= 1.2
        d_o = s.oracle.signed_distance(s.problem, q)
        qt = torch.from_numpy(q.astype(np.float32)).cuda()
        dt = torch.zeros(q.shape[0], dtype=torch.float32, device="cuda")
        lib.cp_signed_distance(s.h, qt, q.shape[0], dt)
        d_g = dt.cpu().numpy()
        # the oracle is evaluated at the float32-rounded configuration for a like-for-like check
        d_o32 = s.oracle.signed_distance(s.problem, q.astype(np.float32).astype(np.float64))
        assert np.max(np.abs(d_g - d_o32)) <= D_TOL
        band = np.abs(d_o32) > FLAG_BAND
        np.testing.assert_array_equal((d_g < 0)[band], (d_o32 < 0)[band])
        assert (d_o < 0).sum() > 100 and (d_o > 0).sum() > 100
    finally:
        s.close()


def test_philox_bits(lib):
    """The GPU generator is bit-identical to the oracle's Philox4x32-10."""
    import oracle
    import torch
    g = np.random.default_rng(11)
    ctr = g.integers(0, 2 ** 32, size=(5000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0], ctr[1] = 0, 0xFFFFFFFF
    for key in (0, 0xFFFFFFFFFFFFFFFF, 0x1234567890ABCDEF):
        want = oracle.philox4x32_10(ctr, (key & 0xFFFFFFFF, key >> 32))
        c = torch.from_numpy(ctr.view(np.int32)).cuda()
        out = torch.zeros_like(c)
        lib.cp_philox4x32_10(c, key, ctr.shape[0], out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), want)


def test_staging_wait_runs_out_and_reports(lib, crane):
    """Failure detection without a fault: the evaluation kernel is told to issue no staging
    copy, so its bounded mbarrier wait runs out (about a second); the CTAs record the
    timeout and leave with nothing in flight, the host reads CP_ERR_TIMEOUT, and the context
    stays usable for the next planner."""
    import time
    import torch
    from paper_2503_14160_gb300 import workloads
    q0, qd = endpoints("single_small")
    scene = _scene("single_small")
    xi = workloads.random_candidates(q0, qd, 4, 32, seed=2)
    model = lib.make_model(crane)
    params = lib.make_params(32, 4, 8, debug_withhold_staging=1)
    bad = lib.Planner(crane, scene, params)
    try:
        lib.cp_set_endpoints(bad.handle, q0, qd)
        x = torch.from_numpy(xi).cuda()
        J = torch.zeros(32, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        lib.cp_evaluate(bad.handle, x, 32, J)
        with pytest.raises(lib.CranePlanError) as e:
            lib.cp_synchronize(bad.handle)
        assert e.value.status == -3
        assert time.perf_counter() - t0 < 30.0
        lib.cp_synchronize(bad.handle)          # the report is cleared once read
    finally:
        bad.close()
    s = Setup(crane, scene, N=32, K=4, S=8)
    try:
        check_eval(s, xi, q0, qd)               # the device keeps working
    finally:
        s.close()


def test_alu_peak_probes(lib):
    """The FMA-pipe probes return plausible rates: FP32 within the part's nominal
    152 SMs x 128 lanes x 2 x 2.07 GHz = 80.5 TFLOP/s, FP64 well below it."""
    p = lib.cp_alu_peaks()
    assert 10.0 < p["fp32_tflops"] < 81.0
    assert 0.05 < p["fp64_tflops"] < p["fp32_tflops"]

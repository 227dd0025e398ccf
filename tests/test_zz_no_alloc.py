"""cp_evaluate_static: candidate evaluation for callers that may not allocate GPU memory
while they run (a real-time control loop, where cudaMalloc can stall the device for an
unbounded time, or a plug-in whose host application owns all device memory). It runs the
planner's own evaluation kernels on a fixed library scratch, so its results must equal
cp_evaluate's bit for bit, call after call, and meet the oracle's tolerances; once the
kernels are loaded a call must take no device memory; a staging wait that runs out must
show in the results.

This file is collected last so that a run stopping at its first failure has already run
every other test."""
import numpy as np
import pytest

from helpers import D_TOL, FLAG_BAND, Setup, cost_tolerance, endpoints

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


def _scene(name, n_cyl=None):
    from paper_2503_14160_gb300 import workloads
    sc = workloads.make_scene(workloads.WORKLOADS[name])
    cyl = sc.cylinders
    if n_cyl is not None:
        cyl = cyl[np.argsort(np.hypot(cyl[:, 0], cyl[:, 1]), kind="stable")[:n_cyl]]
    return workloads.Scene(cyl, sc.boxes[:20])


class _Buffers:
    """Device inputs and outputs of one static call, allocated before it."""

    def __init__(self, scene, xi):
        import torch
        self.cyl = torch.from_numpy(np.ascontiguousarray(scene.cylinders)).cuda()
        self.box = torch.from_numpy(np.ascontiguousarray(scene.boxes)).cuda()
        self.xi = torch.from_numpy(np.ascontiguousarray(xi, np.float32)).cuda()
        n = xi.shape[0]
        self.J = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        self.flag = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        self.terms = torch.zeros(n, 5, dtype=torch.float64, device="cuda")

    def results(self):
        return self.J.cpu().numpy(), self.flag.cpu().numpy(), self.terms.cpu().numpy()


def _static_call(cp, model, scene, K, S, q0, qd, b):
    cp.cp_evaluate_static(model, b.cyl, scene.n_cyl, b.box, scene.n_box, K, S, 100.0, 100.0, 1.0,
                          q0, qd, b.xi, b.xi.shape[0], b.J, b.flag, b.terms)


CASES = [("single_small", None, 8, 32, 256, 1), ("dense_forest", 300, 5, 7, 37, 2)]


def test_static_evaluation_equals_planner_twice(lib):
    """Two calls in a row with different sizes: J, flags and terms equal cp_evaluate's bit
    for bit (the same kernels on the same inputs; the obstacle order does not change a
    minimum of exact distances), and the first case also meets the oracle's tolerances."""
    import torch
    from paper_2503_14160_gb300 import workloads
    crane = workloads.forestry_crane()
    model = lib.make_model(crane)
    for c, (name, n_cyl, K, S, n, seed) in enumerate(CASES):
        scene = _scene(name, n_cyl)
        q0, qd = endpoints(name)
        xi = workloads.random_candidates(q0, qd, K, n, seed=seed)
        b = _Buffers(scene, xi)
        _static_call(lib, model, scene, K, S, q0, qd, b)
        torch.cuda.synchronize()
        Js, fs, ts = b.results()
        s = Setup(crane, scene, N=n, K=K, S=S)
        try:
            g = s.evaluate(xi, q0, qd)
            if c == 0:
                o = s.oracle.evaluate(s.problem, xi.astype(np.float64), q0, qd, with_distances=True)
        finally:
            s.close()
        np.testing.assert_array_equal(Js, g["J"])
        np.testing.assert_array_equal(fs, g["flag"])
        np.testing.assert_array_equal(ts, g["terms"])
        if c == 0:
            d = o.d[:, 1:]
            n_near = (d < D_TOL).sum(axis=1)
            assert np.all(np.abs(Js - o.J) <= cost_tolerance(o.J, n_near))
            clean = ~(np.abs(d) <= FLAG_BAND).any(axis=1)
            np.testing.assert_array_equal(fs[clean], o.flag[clean])
            assert (d < 0).any() and (d > 0).any()          # both sides of contact


def test_static_evaluation_takes_no_device_memory(lib):
    """After a first call has loaded the kernels and looked up the scratch address, further
    calls leave the device's free memory unchanged: nothing is allocated per call."""
    import torch
    from paper_2503_14160_gb300 import workloads
    crane = workloads.forestry_crane()
    model = lib.make_model(crane)
    name, n_cyl, K, S, n, seed = CASES[0]
    scene = _scene(name, n_cyl)
    q0, qd = endpoints(name)
    b = _Buffers(scene, workloads.random_candidates(q0, qd, K, n, seed=seed))
    _static_call(lib, model, scene, K, S, q0, qd, b)
    torch.cuda.synchronize()
    first = b.results()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _static_call(lib, model, scene, K, S, q0, qd, b)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for a, c in zip(first, b.results()):
        np.testing.assert_array_equal(a, c)


def test_static_evaluation_staging_timeout_shows_in_results(lib):
    """With the staging copy withheld (test hook) the bounded wait runs out on the device;
    every J of that call is NaN and every flag 1, and the next call is correct again."""
    import torch
    from paper_2503_14160_gb300 import workloads
    crane = workloads.forestry_crane()
    model = lib.make_model(crane)
    name, n_cyl, K, S, n, seed = CASES[0]
    scene = _scene(name, n_cyl)
    q0, qd = endpoints(name)
    b = _Buffers(scene, workloads.random_candidates(q0, qd, K, n, seed=seed))
    _static_call(lib, model, scene, K, S, q0, qd, b)
    torch.cuda.synchronize()
    good = b.results()
    lib.cp_debug_static_withhold_staging(True)
    try:
        _static_call(lib, model, scene, K, S, q0, qd, b)
        torch.cuda.synchronize()
    finally:
        lib.cp_debug_static_withhold_staging(False)
    J, f, t = b.results()
    assert np.isnan(J).all() and (f == 1).all() and np.isnan(t[:, :4]).all()
    _static_call(lib, model, scene, K, S, q0, qd, b)
    torch.cuda.synchronize()
    for a, c in zip(good, b.results()):
        np.testing.assert_array_equal(a, c)


def test_static_evaluation_rejects_oversize(lib):
    """A call whose work-item sums would not fit the fixed scratch is refused before any
    launch, with a message that says how much it needs. The buffers passed are of the full
    size, so that no path of the call could read or write outside them."""
    import torch
    from paper_2503_14160_gb300 import workloads
    model = lib.make_model(workloads.forestry_crane())
    n, K, S = 1_200_000, 32, 128          # 1.2M items of 36 bytes: about 43 MB of item sums
    xi = torch.zeros(n, K, 4, device="cuda")
    J = torch.zeros(n, dtype=torch.float64, device="cuda")
    empty = torch.zeros(0, 5, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.CranePlanError) as e:
        lib.cp_evaluate_static(model, empty, 0, empty, 0, K, S, 100.0, 100.0, 1.0,
                               np.zeros(4), np.ones(4), xi, n, J)
    assert e.value.status == -1 and "scratch" in str(e.value)

"""GPU parity of the convex-hull collision check (Sec. 3.1; link boxes against boxes and
circumscribed octagonal prisms by separating axes) with the FP64 oracle in oracle/hulls.py.

Tolerance: the depth is max(0, smallest overlap), continuous in the geometry, so the FP32
kernel's error is that of its overlaps: hull corners placed by FP32 kinematics over a 10 m
lever (~1e-6 m) and a few FP32 operations per axis; 2e-5 m, as for the sphere distances.
"""
import numpy as np
import pytest

from helpers import Setup

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def lib():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


def _run(lib, s, q, hulls=None):
    import torch
    qt = torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
    pen = torch.full((max(len(q), 1),), -1.0, device="cuda")
    lib.cp_hull_penetration(s.h, qt, len(q), pen, hulls)
    torch.cuda.synchronize()
    return pen.cpu().numpy()[:len(q)].astype(np.float64)


@pytest.mark.parametrize("name,n", [("single_large", 400), ("dense_forest", 120)])
def test_matches_oracle(lib, crane, name, n):
    import hulls
    from paper_2503_14160_gb300 import workloads
    s = Setup(crane, workloads.make_scene(workloads.WORKLOADS[name]), N=4, K=2, S=2)
    try:
        g = workloads.rng(0, workloads.STREAM_TEST, 5)
        q = workloads.uniform_configurations(crane, g, n)
        q[: n // 10] *= 1.2   # some beyond the limits
        q32 = q.astype(np.float32).astype(np.float64)
        got = _run(lib, s, q32)
        want = hulls.penetration_batch(s.problem, q32)
        np.testing.assert_allclose(got, want, rtol=0, atol=TOL)
        assert (want > 1e-3).sum() > n // 10 and (want == 0).sum() > n // 10
    finally:
        s.close()


def test_custom_hulls_and_free_space(lib, crane):
    import hulls
    from paper_2503_14160_gb300 import workloads
    s = Setup(crane, workloads.make_scene(workloads.WORKLOADS["single_small"]), N=4, K=2, S=2)
    try:
        g = workloads.rng(1, workloads.STREAM_TEST, 6)
        q = workloads.uniform_configurations(crane, g, 300).astype(np.float32).astype(np.float64)
        big = hulls.Hulls(w=(0.35, 0.3, 0.25), h=(0.3, 0.3, 0.2), pad=0.3, grapple_w=0.4, grapple_len=1.5)
        hm = lib.make_hull_model(big.w, big.h, big.pad, big.grapple_w, big.grapple_len)
        got_big = _run(lib, s, q, hm)
        np.testing.assert_allclose(got_big, hulls.penetration_batch(s.problem, q, big), rtol=0, atol=TOL)
        got = _run(lib, s, q)
        assert np.all(got_big >= got - TOL)   # larger hulls penetrate at least as deep
        assert (got_big > got + 1e-3).sum() > 10
    finally:
        s.close()
    e = Setup(crane, workloads.empty_scene(), N=4, K=2, S=2)
    try:
        np.testing.assert_array_equal(_run(lib, e, q), 0.0)
    finally:
        e.close()


def test_edge_cases(lib, crane):
    import torch
    from paper_2503_14160_gb300 import workloads
    s = Setup(crane, workloads.empty_scene(), N=4, K=2, S=2)
    try:
        q = torch.zeros(1, 4, device="cuda")
        pen = torch.zeros(1, device="cuda")
        lib.cp_hull_penetration(s.h, q, 0, pen)
        for bad in (dict(w=(0.0, 0.2, 0.2)), dict(pad=-1.0), dict(grapple_len=0.0)):
            with pytest.raises(Exception):
                lib.cp_hull_penetration(s.h, q, 1, pen, lib.make_hull_model(**bad))
        with pytest.raises(Exception):
            lib.cp_hull_penetration(s.h, q, -1, pen)
    finally:
        s.close()

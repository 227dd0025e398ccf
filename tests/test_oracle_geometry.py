"""Pins of the oracle's kinematics and signed distances against closed forms, invariants
and brute force (Sec. 2 Eq. FK with the chain described in the golden file; Sec. 3.1)."""
import json
import math
import os

import numpy as np
import pytest

from conftest import GOLDEN

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def empty_problem(oracle, crane):
    from paper_2503_14160_gb300 import workloads
    return oracle.Problem(crane, workloads.empty_scene(), oracle.CostParams(K=4, S=8))


def test_fk_closed_forms(oracle, empty_problem):
    cases = json.load(open(os.path.join(GOLDEN, "fk_cases.json")))
    for case in cases["cases"]:
        _, J, T = oracle.fk(empty_problem, case["q"])
        np.testing.assert_allclose(J, case["J"], atol=1e-12, err_msg=case["why"])
        np.testing.assert_allclose(T, case["T"], atol=1e-12, err_msg=case["why"])
    z = cases["spheres_at_zero"]
    c, _, _ = oracle.fk(empty_problem, z["q"])
    np.testing.assert_allclose(c, z["centres"], atol=1e-12)


def test_fk_invariants_random(oracle, empty_problem, crane):
    """Link lengths, the jib angle and the plumb grapple hold at any configuration."""
    g = np.random.default_rng(1)
    lo, hi = np.array(crane.q_min), np.array(crane.q_max)
    for _ in range(200):
        q = lo + (hi - lo) * g.random(4)
        c, J, T = oracle.fk(empty_problem, q)
        assert abs(np.linalg.norm(J) - 4.0) < 1e-12
        assert abs(np.linalg.norm(T - J) - (3.5 + q[3])) < 1e-12
        eb = J / 4.0
        ej = (T - J) / (3.5 + q[3])
        assert abs(eb @ ej - math.cos(q[2])) < 1e-12          # angle between boom and jib
        assert abs(eb[2] - math.sin(q[1])) < 1e-12            # boom elevation
        assert abs(math.atan2(eb[1], eb[0]) - q[0]) < 1e-9 or abs(math.cos(q[1])) < 1e-9
        # boom and jib lie in the vertical plane through the slew direction
        nrm = np.array([-math.sin(q[0]), math.cos(q[0]), 0.0])
        assert abs(nrm @ J) < 1e-12 and abs(nrm @ T) < 1e-12
        # grapple spheres are plumb below the tip
        np.testing.assert_allclose(c[10], T - [0, 0, 0.5], atol=1e-12)
        np.testing.assert_allclose(c[11], T - [0, 0, 1.0], atol=1e-12)
        # telescope spheres: J + (3.5 + t q4) e_j for t = 0.5, 1.0
        np.testing.assert_allclose(c[8], J + (3.5 + 0.5 * q[3]) * ej, atol=1e-12)
        np.testing.assert_allclose(c[9], T, atol=1e-12)


CYL = [1.0, -2.0, 0.5, 0.0, 15.0]   # cx, cy, R, z_lo, z_hi


@pytest.mark.parametrize("p,expected,region", [
    ([1.0 + 2.0, -2.0, 5.0], 1.5, "side: rho - R"),
    ([1.0, -2.0 + 0.3, 5.0], -0.2, "inside, nearest the side: rho - R"),
    ([1.0, -2.0, 17.0], 2.0, "above the top cap: z - z_hi"),
    ([1.0 + 0.1, -2.0, 14.5], -0.4, "inside, nearest the side"),
    ([1.0, -2.0, 14.9], -0.1, "inside, nearest the top cap"),
    ([1.0, -2.0, -0.75], 0.75, "below the bottom cap"),
    ([1.0 + 0.5 + 3.0, -2.0, 15.0 + 4.0], 5.0, "outside the rim: hypot(3, 4)"),
    ([1.0 + 0.5 + 0.3, -2.0, -0.4], 0.5, "outside the bottom rim: hypot(0.3, 0.4)"),
    ([1.0, -2.0, 7.5], -0.5, "on the axis at mid height: -R"),
])
def test_sdf_cylinder_regions(oracle, p, expected, region):
    assert oracle.sdf_cylinder(p, CYL) == pytest.approx(expected, abs=1e-12), region


BOX = [0.0, 0.0, 0.0, 2.0, 4.0, 1.0]   # lo xyz, hi xyz


@pytest.mark.parametrize("p,expected,region", [
    ([3.0, 2.0, 0.5], 1.0, "face +x"),
    ([1.0, -0.5, 0.5], 0.5, "face -y"),
    ([1.0, 2.0, 3.0], 2.0, "face +z"),
    ([5.0, 8.0, 0.5], 5.0, "edge: hypot(3, 4)"),
    ([4.0, 6.0, 3.0], math.sqrt(12.0), "corner"),
    ([1.0, 2.0, 0.5], -0.5, "centre: minus the smallest half extent"),
    ([1.9, 2.0, 0.5], -0.1, "inside near +x"),
])
def test_sdf_box_regions(oracle, p, expected, region):
    assert oracle.sdf_box(p, BOX) == pytest.approx(expected, abs=1e-12), region


def _surface_distance_cylinder(p, cyl, n=400):
    """Brute-force unsigned distance to the cylinder surface by dense sampling."""
    cx, cy, R, z0, z1 = cyl
    th = np.linspace(0, 2 * np.pi, n, endpoint=False)
    zs = np.linspace(z0, z1, n)
    side = np.stack(np.meshgrid(th, zs), -1).reshape(-1, 2)
    pts = [np.stack([cx + R * np.cos(side[:, 0]), cy + R * np.sin(side[:, 0]), side[:, 1]], 1)]
    rr = np.linspace(0, R, n // 4)
    cap = np.stack(np.meshgrid(th, rr), -1).reshape(-1, 2)
    for zc in (z0, z1):
        pts.append(np.stack([cx + cap[:, 1] * np.cos(cap[:, 0]), cy + cap[:, 1] * np.sin(cap[:, 0]),
                             np.full(cap.shape[0], zc)], 1))
    pts = np.concatenate(pts)
    return np.min(np.linalg.norm(pts - np.asarray(p)[None, :], axis=1))


def test_sdf_cylinder_brute_force(oracle):
    """|d| equals the distance to the surface found by dense sampling; the sign is
    negative exactly inside."""
    cyl = [0.3, 0.2, 0.4, 0.0, 2.0]
    g = np.random.default_rng(3)
    for _ in range(60):
        p = g.uniform([-1.0, -1.0, -1.0], [1.5, 1.5, 3.0])
        d = oracle.sdf_cylinder(p, cyl)
        bf = _surface_distance_cylinder(p, cyl)
        inside = math.hypot(p[0] - 0.3, p[1] - 0.2) < 0.4 and 0.0 < p[2] < 2.0
        assert (d < 0) == inside
        assert abs(abs(d) - bf) < 1.5e-2   # sampling resolution


def test_sdf_eikonal(oracle):
    """Away from the medial surface a signed distance has unit gradient."""
    g = np.random.default_rng(4)
    h = 1e-6
    for f, shape in ((oracle.sdf_cylinder, [0.0, 0.0, 0.5, 0.0, 3.0]),
                     (oracle.sdf_box, [-1.0, -0.5, 0.0, 1.0, 0.5, 2.0])):
        n_ok = 0
        for _ in range(200):
            p = g.uniform(-3, 5, size=3)
            d = f(p, shape)
            if abs(d) < 0.05:
                continue
            grad = np.array([(f(p + h * e, shape) - f(p - h * e, shape)) / (2 * h) for e in np.eye(3)])
            if d > 0:   # outside: the distance field is smooth off the shape
                assert abs(np.linalg.norm(grad) - 1.0) < 1e-5
                n_ok += 1
        assert n_ok > 50


def test_signed_distance_tiny_scene(oracle, crane):
    """d(q) on a one-cylinder scene, worked out by hand at q = 0 (all spheres on +x)."""
    from paper_2503_14160_gb300 import workloads
    # cylinder of radius 0.2 at (5, 0.3): nearest sphere is the jib sphere at x = 5.3125;
    # horizontal distance hypot(0.3125, 0.3); minus R + r = 0.45.
    sc = workloads.Scene(np.array([[5.0, 0.3, 0.2, 0.0, 15.0]]), np.zeros((0, 6)))
    pb = oracle.Problem(crane, sc, oracle.CostParams(K=4, S=8))
    d = oracle.signed_distance(pb, [[0.0, 0.0, 0.0, 0.0]])[0]
    assert d == pytest.approx(math.hypot(0.3125, 0.3) - 0.45, abs=1e-12)
    # raising the boom to vertical lifts every sphere off the x axis: the nearest is
    # then the boom sphere row at x = 0 ... the jib sphere J + 3.0625 e_j with e_j = +x
    # at height 4: horizontal distance to the axis hypot(3.0625 - 5, 0.3) but z = 4 is
    # within the cylinder's height, so d = hypot(1.9375, 0.3) - 0.45 ... unless a
    # telescope sphere is nearer: T = (3.5, 0, 4) -> hypot(1.5, 0.3) - 0.45.
    d2 = oracle.signed_distance(pb, [[0.0, math.pi / 2, -math.pi / 2, 0.0]])[0]
    assert d2 == pytest.approx(math.hypot(1.5, 0.3) - 0.45, abs=1e-12)
    # a box as the only obstacle: grapple sphere at (7.5, 0, -1) above a box top at z=-1.5
    sc2 = workloads.Scene(np.zeros((0, 5)), np.array([[7.0, -0.5, -3.0, 8.0, 0.5, -1.5]]))
    pb2 = oracle.Problem(crane, sc2, oracle.CostParams(K=4, S=8))
    d3 = oracle.signed_distance(pb2, [[0.0, 0.0, 0.0, 0.0]])[0]
    assert d3 == pytest.approx(0.5 - 0.25, abs=1e-12)


def test_signed_distance_empty_scene(oracle, empty_problem):
    assert np.isinf(oracle.signed_distance(empty_problem, [[0.1, 0.2, -0.5, 1.0]])[0])

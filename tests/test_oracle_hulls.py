"""Pins of the convex-hull collision oracle (oracle/hulls.py): the separating-axis depth
against a linear-programming separation test that knows nothing of the axes (disjoint
exactly when SAT says so; the depth the shortest translation that separates, along its
axis and against random other directions), the closed form of axis-aligned boxes, the link
boxes at q = 0, and the octagonal prism containing its cylinder."""
import math

import numpy as np
import pytest
from scipy.optimize import linprog

from helpers import ROOT  # noqa: F401  (puts the oracle on sys.path)


@pytest.fixture(scope="module")
def hl():
    import hulls
    return hulls


def separated(va, vb):
    """True when a plane a.x = b strictly separates the vertex sets (margin 1e-9 after
    scaling a.x - b <= -1 on A and >= 1 on B): an LP feasibility problem."""
    na, nb = len(va), len(vb)
    A = np.zeros((na + nb, 4))
    A[:na, :3], A[:na, 3] = va, -1.0
    A[na:, :3], A[na:, 3] = -vb, 1.0
    ub = -np.ones(na + nb)
    res = linprog(np.zeros(4), A_ub=A, b_ub=ub, bounds=[(None, None)] * 4, method="highs")
    return res.status == 0


def random_rotation(g):
    q, r = np.linalg.qr(g.normal(size=(3, 3)))
    return (q * np.sign(np.diag(r))).T   # rows: axes


def random_pair(hl, g, kind):
    axes = random_rotation(g)
    half = g.uniform(0.1, 1.0, 3)
    centre = g.uniform(-1.0, 1.0, 3)
    if kind == "box":
        lo = g.uniform(-1.2, 0.2, 3)
        box = np.concatenate([lo, lo + g.uniform(0.2, 1.5, 3)])
        vb = hl.box_vertices(0.5 * (box[:3] + box[3:]), np.eye(3), 0.5 * (box[3:] - box[:3]))
        pen = hl.pen_boxes(centre, axes, half, [box])[0]
        ax = hl.box_axes(axes)
    else:
        cyl = np.array([g.uniform(-0.8, 0.8), g.uniform(-0.8, 0.8), g.uniform(0.1, 0.6), g.uniform(-1.5, -0.2),
                        g.uniform(0.2, 1.5)])
        vb = hl.prism_vertices(cyl)
        pen = hl.pen_cylinders(centre, axes, half, [cyl])[0]
        ax = hl.prism_axes(axes)
    return centre, axes, half, vb, pen, ax


@pytest.mark.parametrize("kind", ["box", "prism"])
def test_disjoint_exactly_when_sat_says(hl, kind):
    g = np.random.default_rng(1 if kind == "box" else 2)
    n_sep = n_hit = 0
    for _ in range(150):
        centre, axes, half, vb, pen, _ = random_pair(hl, g, kind)
        va = hl.box_vertices(centre, axes, half)
        if pen > 1e-7:
            assert not separated(va, vb)
            n_hit += 1
        elif pen == 0.0:
            assert separated(va, vb) or abs(hl.min_overlap_axis(centre, axes, half, vb, hl.box_axes(axes) if kind == "box" else hl.prism_axes(axes))[0]) < 1e-7
            n_sep += 1
    assert n_sep > 20 and n_hit > 20


@pytest.mark.parametrize("kind", ["box", "prism"])
def test_depth_is_the_shortest_translation(hl, kind):
    g = np.random.default_rng(3 if kind == "box" else 4)
    done = 0
    while done < 25:
        centre, axes, half, vb, pen, ax = random_pair(hl, g, kind)
        if pen < 1e-3:
            continue
        o, L = hl.min_overlap_axis(centre, axes, half, vb, ax)
        assert o == pytest.approx(pen, abs=1e-12)
        # moving A by a hair more than the depth along its axis separates the pair ...
        assert separated(hl.box_vertices(centre + (pen + 1e-6) * L, axes, half), vb)
        # ... a hair less does not, and nor does a shorter move in any other direction
        assert not separated(hl.box_vertices(centre + (pen - 1e-6) * L, axes, half), vb)
        for u in g.normal(size=(10, 3)):
            u /= np.linalg.norm(u)
            assert not separated(hl.box_vertices(centre + 0.995 * pen * u, axes, half), vb)
        done += 1


def test_axis_aligned_boxes_closed_form(hl):
    g = np.random.default_rng(5)
    for _ in range(200):
        ca, ha = g.uniform(-1, 1, 3), g.uniform(0.1, 1, 3)
        lo = g.uniform(-1.5, 0.5, 3)
        hi = lo + g.uniform(0.1, 1.5, 3)
        want = max(0.0, float(np.min(ha + 0.5 * (hi - lo) - np.abs(0.5 * (lo + hi) - ca))))
        assert hl.pen_boxes(ca, np.eye(3), ha, [np.concatenate([lo, hi])])[0] == pytest.approx(want, abs=1e-12)


def test_link_boxes_at_zero(hl, oracle, crane):
    from paper_2503_14160_gb300 import workloads
    pb = oracle.Problem(crane, workloads.empty_scene(), oracle.CostParams(K=1, S=1))
    H = hl.Hulls()
    q4 = 0.7
    boxes = hl.link_boxes(pb, [0.0, 0.0, 0.0, q4], H)
    Lb, Lj = crane.boom_len, crane.jib_len
    np.testing.assert_allclose(boxes[0][0], [Lb / 2, 0, crane.base_z], atol=1e-14)
    np.testing.assert_allclose(boxes[1][0], [Lb + Lj / 2, 0, crane.base_z], atol=1e-14)
    np.testing.assert_allclose(boxes[2][0], [Lb + Lj + q4 / 2, 0, crane.base_z], atol=1e-14)
    np.testing.assert_allclose(boxes[3][0], [Lb + Lj + q4, 0, crane.base_z - H.grapple_len / 2], atol=1e-14)
    np.testing.assert_allclose(boxes[0][1], np.eye(3), atol=1e-15)
    np.testing.assert_allclose(boxes[2][2], [q4 / 2 + H.pad, H.w[2], H.h[2]], atol=1e-15)
    # q1 = pi/2 turns every box about z onto the y axis
    turned = hl.link_boxes(pb, [math.pi / 2, 0.0, 0.0, q4], H)
    np.testing.assert_allclose(turned[1][0], [0, Lb + Lj / 2, crane.base_z], atol=1e-12)


def test_prism_contains_its_cylinder(hl):
    g = np.random.default_rng(6)
    cyl = np.array([0.3, -0.2, 0.4, 0.0, 2.0])
    vb = hl.prism_vertices(cyl)
    for t in g.uniform(0, 2 * math.pi, 200):
        p = np.array([cyl[0] + cyl[2] * math.cos(t), cyl[1] + cyl[2] * math.sin(t), g.uniform(0, 2)])
        # inside the hull of the prism's vertices: not separable from it
        assert not separated(p[None, :] + 1e-12, vb)
        # and on the prism's faces at most at the apothem
        assert np.max(np.abs((p[:2] - cyl[:2]) @ hl.OCT_DIRS[:, :2].T)) <= cyl[2] + 1e-12


def test_checkpoint_configurations_are_the_costs(hl, oracle, crane):
    """The checkpoints of the hull-form cost are those of the oracle's path cost: the sphere
    model's penetration summed over them is the oracle's J_c."""
    from paper_2503_14160_gb300 import workloads
    scene = workloads.make_scene(workloads.WORKLOADS["single_small"])
    pb = oracle.Problem(crane, scene, oracle.CostParams(K=3, S=5))
    q0, qd = np.array([0.3, 0.2, -1.0, 0.4]), np.array([-2.0, 0.9, -0.6, 1.8])
    xi = workloads.random_candidates(q0, qd, 3, 6, seed=2)
    base = oracle.evaluate(pb, xi, q0, qd)
    for i in range(6):
        qs = hl.checkpoint_configurations(pb, xi[i], q0, qd)
        assert len(qs) == (3 + 3) * 5
        np.testing.assert_allclose(qs[-1], qd, atol=1e-12)
        pen = np.maximum(0.0, -oracle.signed_distance(pb, qs))
        assert pb.cost.lambda_c * pen.sum() == pytest.approx(base.Jc[i], rel=1e-12, abs=1e-12)

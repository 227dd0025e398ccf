"""FP64 oracle of the convex-hull collision model (arXiv 2503.14160, Sec. 3.1: the crane's
links as convex hulls checked against the obstacles by the separating axis theorem) -- TEST
INFRASTRUCTURE, like the rest of oracle/.

The paper's 32 crane meshes are not available, so synthetic hulls stand in: each link is an
oriented box (OBB) placed by the crane kinematics of the C oracle (`oracle.fk`):
    boom       centre O + (L_b / 2) e_b, axes (e_b, n, e_b x n), half extents
               (L_b / 2 + pad, w, h)
    jib        centre J + (L_j / 2) e_j, axes (e_j, n, e_j x n)
    telescope  centre J + (L_j + q4+ / 2) e_j, q4+ = max(q4, 0), half length q4+ / 2 + pad
    grapple    centre T - (0, 0, g / 2), axes ((c1, s1, 0), n, z), half (w_g, w_g, g / 2)
with n = (-sin q1, cos q1, 0) the normal of the crane's vertical plane. Obstacles: the
axis-aligned boxes as they are, and each vertical cylinder as the regular octagonal prism
that circumscribes it (apothem R, side normals at multiples of 45 degrees, the cylinder's
height range).

For two centrally symmetric convex polytopes the overlap along a unit axis L is
    o(L) = r_A(L) + r_B(L) - |(c_B - c_A) . L|
with r the support half-width. They are disjoint iff o(L) < 0 for some L among the face
normals of both and the cross products of their edge directions, and otherwise the smallest
o(L) over that set is the penetration depth (the shortest translation that separates them).
The hull penetration of a configuration is the largest depth over links and obstacles, 0
when every pair is disjoint.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

import oracle as _o


@dataclasses.dataclass(frozen=True)
class Hulls:
    """Half extents (m) of the four link boxes across their axis (w: along n, h: in the
    plane), the end padding of the three arm boxes, and the grapple box."""
    w: tuple = (0.2, 0.2, 0.15)     # boom, jib, telescope
    h: tuple = (0.2, 0.2, 0.15)
    pad: float = 0.2
    grapple_w: float = 0.25
    grapple_len: float = 1.0


OCT_C = math.cos(math.pi / 8.0)
# unit directions of the octagon's side normals and, for the same angles, its edge directions
OCT_DIRS = np.array([[math.cos(k * math.pi / 4), math.sin(k * math.pi / 4), 0.0] for k in range(4)])
# vertex directions (half-way between the side normals), circumradius R / cos(pi / 8)
OCT_VERTS = np.array([[math.cos((k + 0.5) * math.pi / 4), math.sin((k + 0.5) * math.pi / 4)] for k in range(8)])


def link_boxes(problem, q, hulls: Hulls):
    """[(centre[3], axes[3][3] (rows), half[3])] of the four link boxes at configuration q."""
    q = np.asarray(q, dtype=np.float64)
    m = problem.model_py
    _, J, T = _o.fk(problem, q)
    c1, s1 = math.cos(q[0]), math.sin(q[0])
    eb = np.array([math.cos(q[1]) * c1, math.cos(q[1]) * s1, math.sin(q[1])])
    a = q[1] + q[2]
    ej = np.array([math.cos(a) * c1, math.cos(a) * s1, math.sin(a)])
    n = np.array([-s1, c1, 0.0])
    O = np.array([0.0, 0.0, m.base_z])
    q4p = max(q[3], 0.0)
    out = []
    for centre, e, half_len, w, h in (
            (O + 0.5 * m.boom_len * eb, eb, 0.5 * m.boom_len + hulls.pad, hulls.w[0], hulls.h[0]),
            (J + 0.5 * m.jib_len * ej, ej, 0.5 * m.jib_len + hulls.pad, hulls.w[1], hulls.h[1]),
            (J + (m.jib_len + 0.5 * q4p) * ej, ej, 0.5 * q4p + hulls.pad, hulls.w[2], hulls.h[2])):
        out.append((centre, np.array([e, n, np.cross(e, n)]), np.array([half_len, w, h])))
    g = hulls.grapple_len
    out.append((T - np.array([0.0, 0.0, 0.5 * g]), np.array([[c1, s1, 0.0], n, [0.0, 0.0, 1.0]]),
                np.array([hulls.grapple_w, hulls.grapple_w, 0.5 * g])))
    return out


def _unit_axes(vectors):
    """The given axes normalised; near-zero cross products (parallel edges) dropped."""
    v = np.asarray(vectors, dtype=np.float64)
    nrm = np.linalg.norm(v, axis=1)
    keep = nrm > 1e-9
    return v[keep] / nrm[keep][:, None]


def _obb_support(axes, half, L):
    """r_A(L) for unit axes L[k][3]."""
    return np.abs(L @ axes.T) @ half


def box_axes(axes):
    e = np.eye(3)
    cross = [np.cross(u, v) for u in axes for v in e]
    return _unit_axes(np.concatenate([axes, e, np.array(cross)]))


def prism_axes(axes):
    z = np.array([0.0, 0.0, 1.0])
    edge_dirs = np.concatenate([[z], OCT_DIRS])
    cross = [np.cross(u, v) for u in axes for v in edge_dirs]
    return _unit_axes(np.concatenate([axes, [z], OCT_DIRS, np.array(cross)]))


def prism_support(R, half_h, L):
    """r_B(L) of octagonal prisms [M] (apothem R, half height) along unit axes L[k]:
    [k][M]."""
    rc = np.asarray(R) / OCT_C
    xy = np.max(np.abs(L[:, :2] @ OCT_VERTS.T), axis=1)          # [k]
    return np.abs(L[:, 2])[:, None] * np.asarray(half_h)[None, :] + xy[:, None] * rc[None, :]


def pen_boxes(centre, axes, half, boxes):
    """Penetration depth of one OBB against axis-aligned boxes [M][6] (lo, hi): [M]."""
    if len(boxes) == 0:
        return np.zeros(0)
    b = np.asarray(boxes, dtype=np.float64)
    bc, bh = 0.5 * (b[:, :3] + b[:, 3:]), 0.5 * (b[:, 3:] - b[:, :3])
    L = box_axes(axes)
    o = (_obb_support(axes, half, L)[:, None] + np.abs(L) @ bh.T - np.abs((bc - centre) @ L.T).T)
    return np.maximum(0.0, o.min(axis=0))


def pen_cylinders(centre, axes, half, cyl):
    """Penetration depth of one OBB against the octagonal prisms of cylinders [M][5]
    (cx, cy, R, z_lo, z_hi): [M]."""
    if len(cyl) == 0:
        return np.zeros(0)
    c = np.asarray(cyl, dtype=np.float64)
    pc = np.stack([c[:, 0], c[:, 1], 0.5 * (c[:, 3] + c[:, 4])], axis=1)
    L = prism_axes(axes)
    o = (_obb_support(axes, half, L)[:, None] + prism_support(c[:, 2], 0.5 * (c[:, 4] - c[:, 3]), L)
         - np.abs((pc - centre) @ L.T).T)
    return np.maximum(0.0, o.min(axis=0))


def penetration(problem, q, hulls: Hulls = Hulls()) -> float:
    """The hull penetration of configuration q: the largest SAT depth over links and
    obstacles (0 when every pair is disjoint)."""
    best = 0.0
    for centre, axes, half in link_boxes(problem, q, hulls):
        for pen in (pen_cylinders(centre, axes, half, problem.cyl), pen_boxes(centre, axes, half, problem.box)):
            if len(pen):
                best = max(best, float(pen.max()))
    return best


def penetration_batch(problem, qs, hulls: Hulls = Hulls()) -> np.ndarray:
    return np.array([penetration(problem, q, hulls) for q in np.asarray(qs, dtype=np.float64).reshape(-1, 4)])


def min_overlap_axis(centre, axes, half, verts_b, axes_b):
    """(smallest overlap, its unit axis oriented from B's centre towards A's) of one OBB
    and a centrally symmetric polytope given by its vertices, over the candidate axes
    axes_b (for the pins, with the support of B taken from its vertices)."""
    cb = verts_b.mean(axis=0)
    rb = np.max(np.abs((verts_b - cb) @ axes_b.T), axis=0)
    d = (centre - cb) @ axes_b.T
    o = _obb_support(axes, half, axes_b) + rb - np.abs(d)
    k = int(np.argmin(o))
    return float(o[k]), axes_b[k] * (1.0 if d[k] >= 0.0 else -1.0)


def checkpoint_configurations(problem, xi, q0, qd):
    """q(s_k), k = 1..n_s, of one candidate xi[K][4] (the spline of the oracle's cost:
    control points q0 x4, xi, qd x4, tau(s) = 4 + (K + 3) s, s_k = k / n_s)."""
    K, S = problem.cost.K, problem.cost.S
    n_s = (K + 3) * S
    P = np.concatenate([np.tile(_o._c64(q0), (4, 1)), np.asarray(xi, dtype=np.float64).reshape(K, 4),
                        np.tile(_o._c64(qd), (4, 1))])
    return np.array([_o.bspline(P, 4.0 + (K + 3) * k / n_s) for k in range(1, n_s + 1)])


def evaluate_hulls(problem, xi, q0, qd, hulls: Hulls = Hulls()):
    """Eq. path opt with the hull model's collision term: (J, Jc, pen[n][n_s]) for candidates
    xi[n][K][4]. J_p and J_l are the model-free terms of the oracle's cost;
    J_c = lambda_c sum_k pen(q(s_k)) with pen the hull penetration."""
    c = problem.cost
    base = _o.evaluate(problem, xi, q0, qd)
    xi = np.asarray(xi, dtype=np.float64).reshape(-1, c.K, 4)
    pen = np.array([penetration_batch(problem, checkpoint_configurations(problem, x, q0, qd), hulls) for x in xi])
    Jc = c.lambda_c * pen.sum(axis=1)
    J = base.Jp + c.w_c * Jc + c.w_l * base.Jl
    return J, Jc, pen


# ---------------------------------------------------------------- geometry used by the pins

def box_vertices(centre, axes, half):
    s = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], dtype=np.float64)
    return centre[None, :] + (s * half[None, :]) @ axes


def prism_vertices(cyl):
    cx, cy, R, zlo, zhi = cyl
    rc = R / OCT_C
    ring = np.array([[cx + rc * v[0], cy + rc * v[1]] for v in OCT_VERTS])
    return np.concatenate([np.column_stack([ring, np.full(8, zlo)]), np.column_stack([ring, np.full(8, zhi)])])

"""Seeded synthetic inputs: the crane model description, forest scenes, start/goal draws
and random candidate buffers.

This module draws numbers and lays them out; it holds none of the planner's arithmetic
(no kinematics, distances, splines or costs). Both the CUDA path and the FP64 oracle take
their inputs from here. Where an input has to satisfy a property of the method (start and
goal free of collision), the caller passes in the distance function to use.

The paper's benchmark environments (truck trunk, rungs, cluttered obstacles; Sec. 5.2)
and crane meshes are not available, so synthetic crane-and-forest scenes stand in for
them: vertical cylinders ("trees") around the crane base and, for the dense forest,
axis-aligned boxes as terrain.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

# Stream ids folded into the seed of every draw (one independent stream per use).
STREAM_SCENE = 1
STREAM_ENDPOINTS = 2
STREAM_QUERY_SIZES = 3
STREAM_TEST = 7
STREAM_IK_TARGETS = 4


def rng(seed: int, stream: int, *extra: int) -> np.random.Generator:
    """Independent numpy Philox stream for (seed, stream, extra...)."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, stream, *extra])))


# --------------------------------------------------------------------------- crane model

@dataclasses.dataclass(frozen=True)
class Sphere:
    link: int       # 0 boom, 1 jib, 2 telescope, 3 grapple
    offset: float   # placement parameter t along the link (m)
    radius: float   # m


@dataclasses.dataclass(frozen=True)
class CraneModel:
    """The actuated chain of the forestry crane (slew, boom, jib, telescope) with a
    plumb grapple, and the link spheres that bound it.

    Placement of sphere centres (t = offset):
      boom      O + t e_b
      jib       J + t e_j
      telescope J + (jib_len + t q4) e_j
      grapple   T - t z
    with O the slew/boom pivot, J the jib pivot and T the tip.
    """
    base_z: float
    boom_len: float
    jib_len: float
    q_min: tuple
    q_max: tuple
    spheres: tuple


def forestry_crane() -> CraneModel:
    """Slew revolute about z, boom pitch (4.0 m), jib pitch (3.5 m), telescope 0-2.5 m,
    grapple 1.0 m below the tip; 12 link spheres of radius 0.25 m."""
    r = 0.25
    spheres = (
        [Sphere(0, t, r) for t in (0.5, 1.5, 2.5, 3.5)]
        + [Sphere(1, t, r) for t in (0.4375, 1.3125, 2.1875, 3.0625)]
        + [Sphere(2, t, r) for t in (0.5, 1.0)]
        + [Sphere(3, t, r) for t in (0.5, 1.0)]
    )
    return CraneModel(
        base_z=0.0, boom_len=4.0, jib_len=3.5,
        q_min=(-math.pi, -0.3, -2.6, 0.0),
        q_max=(math.pi, 1.3, -0.2, 2.5),
        spheres=tuple(spheres),
    )


# --------------------------------------------------------------------------- scenes

@dataclasses.dataclass
class Scene:
    cylinders: np.ndarray   # float64 [M][5]: cx, cy, R, z_lo, z_hi
    boxes: np.ndarray       # float64 [B][6]: lo xyz, hi xyz

    @property
    def n_cyl(self) -> int:
        return int(self.cylinders.shape[0])

    @property
    def n_box(self) -> int:
        return int(self.boxes.shape[0])


def empty_scene() -> Scene:
    return Scene(np.zeros((0, 5)), np.zeros((0, 6)))


def annulus_cylinders(g: np.random.Generator, m: int, r_in: float, r_out: float,
                      rad_lo: float, rad_hi: float, height: float = 15.0) -> np.ndarray:
    """m vertical cylinders, centres uniform in area over the annulus r_in..r_out around
    the crane base, radii uniform in [rad_lo, rad_hi], from z = 0 to z = height."""
    rho = np.sqrt(g.uniform(r_in * r_in, r_out * r_out, size=m))
    phi = g.uniform(0.0, 2.0 * math.pi, size=m)
    rad = g.uniform(rad_lo, rad_hi, size=m)
    out = np.zeros((m, 5))
    out[:, 0] = rho * np.cos(phi)
    out[:, 1] = rho * np.sin(phi)
    out[:, 2] = rad
    out[:, 3] = 0.0
    out[:, 4] = height
    return out


def poisson_disc_cylinders(g: np.random.Generator, m: int, r_in: float, r_out: float,
                           rad_lo: float, rad_hi: float, spacing: float,
                           height: float = 15.0, max_draws: int = 2_000_000) -> np.ndarray:
    """Dart throwing: area-uniform draws in the annulus, kept when every kept centre is at
    least `spacing` away (checked on a hash grid of cell size `spacing`)."""
    cell = spacing
    grid: Dict[tuple, List[int]] = {}
    pts: List[tuple] = []
    draws = 0
    batch = 4096
    while len(pts) < m and draws < max_draws:
        rho = np.sqrt(g.uniform(r_in * r_in, r_out * r_out, size=batch))
        phi = g.uniform(0.0, 2.0 * math.pi, size=batch)
        xs, ys = rho * np.cos(phi), rho * np.sin(phi)
        for x, y in zip(xs.tolist(), ys.tolist()):
            draws += 1
            cx, cy = int(math.floor(x / cell)), int(math.floor(y / cell))
            ok = True
            for ix in range(cx - 1, cx + 2):
                for iy in range(cy - 1, cy + 2):
                    for idx in grid.get((ix, iy), ()):
                        px, py = pts[idx]
                        if (px - x) ** 2 + (py - y) ** 2 < spacing * spacing:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                grid.setdefault((cx, cy), []).append(len(pts))
                pts.append((x, y))
                if len(pts) == m:
                    break
    if len(pts) < m:
        raise RuntimeError("dart throwing placed %d of %d cylinders" % (len(pts), m))
    rad = g.uniform(rad_lo, rad_hi, size=m)
    out = np.zeros((m, 5))
    out[:, 0:2] = np.asarray(pts)
    out[:, 2] = rad
    out[:, 4] = height
    return out


def annulus_boxes(g: np.random.Generator, m: int, r_in: float, r_out: float,
                  side_lo: float, side_hi: float) -> np.ndarray:
    """m axis-aligned boxes resting on z = 0, centres area-uniform in the annulus, each
    side uniform in [side_lo, side_hi]."""
    rho = np.sqrt(g.uniform(r_in * r_in, r_out * r_out, size=m))
    phi = g.uniform(0.0, 2.0 * math.pi, size=m)
    side = g.uniform(side_lo, side_hi, size=(m, 3))
    cx, cy = rho * np.cos(phi), rho * np.sin(phi)
    out = np.zeros((m, 6))
    out[:, 0] = cx - 0.5 * side[:, 0]
    out[:, 1] = cy - 0.5 * side[:, 1]
    out[:, 2] = 0.0
    out[:, 3] = cx + 0.5 * side[:, 0]
    out[:, 4] = cy + 0.5 * side[:, 1]
    out[:, 5] = side[:, 2]
    return out


# --------------------------------------------------------------------------- workloads

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_candidates: int
    n_waypoints: int
    substeps: int
    iterations: int
    n_cyl: int
    r_in: float
    r_out: float
    rad_lo: float
    rad_hi: float
    spacing: float = 0.0        # >0: Poisson-disc placement
    grid_cell: float = 0.0      # >0: evaluate through the polar obstacle index, rings of this width
    n_box: int = 0
    box_r_in: float = 2.0
    box_r_out: float = 12.0
    box_side_lo: float = 0.5
    box_side_hi: float = 2.0
    seed: int = 0

    @property
    def n_checkpoints(self) -> int:
        return (self.n_waypoints + 3) * self.substeps


WORKLOADS: Dict[str, Workload] = {
    # Plain single query: 20 trees in a 2-8 m annulus; N=256, K=8, S=32, 50 iterations.
    "single_small": Workload("single_small", 256, 8, 32, 50, 20, 2.0, 8.0, 0.1, 0.4),
    # Single large query: 500 trees in a 2-10 m annulus; N=4096, K=16, S=64, 100 iterations;
    # the polar index with rings of 0.5 m (faster here than the broad phase).
    "single_large": Workload("single_large", 4096, 16, 64, 100, 500, 2.0, 10.0, 0.1, 0.4, grid_cell=0.5),
    # Dense forest: 5000 trees (Poisson disc >= 0.8 m, 2-50 m annulus) + 50 boxes;
    # N=65536, K=32, S=128, 200 iterations.
    "dense_forest": Workload("dense_forest", 65536, 32, 128, 200, 5000, 2.0, 50.0, 0.1, 0.5,
                             spacing=0.8, n_box=50, grid_cell=0.5),
    # Differentiable form: 1000 trees in a 2-14 m annulus; N=16384, K=32, S=64.
    "differentiable": Workload("differentiable", 16384, 32, 64, 0, 1000, 2.0, 14.0, 0.1, 0.4),
}


@dataclasses.dataclass(frozen=True)
class BatchQuery:
    n_candidates: int
    n_waypoints: int
    n_cyl: int
    r_out: float


def batch_queries(nq: int = 64, seed: int = 0, n_lo: int = 1024, n_hi: int = 16384,
                  k_lo: int = 8, k_hi: int = 32, m_lo: int = 50, m_hi: int = 3000,
                  density: float = 1.66) -> List[BatchQuery]:
    """Uneven query sizes of the batched serving form: N, K and the cylinder count uniform
    in their ranges; each scene fills an annulus 2..r_out at the given trees per m^2,
    r_out = sqrt(4 + M / (density pi))."""
    g = rng(seed, STREAM_QUERY_SIZES)
    out = []
    for _ in range(nq):
        N = int(g.integers(n_lo, n_hi + 1))
        K = int(g.integers(k_lo, k_hi + 1))
        M = int(g.integers(m_lo, m_hi + 1))
        out.append(BatchQuery(N, K, M, math.sqrt(4.0 + M / (density * math.pi))))
    return out


def batch_scene(bq: BatchQuery, seed: int, q: int) -> Scene:
    g = rng(seed, STREAM_SCENE, 1000 + q)
    return Scene(annulus_cylinders(g, bq.n_cyl, 2.0, bq.r_out, 0.1, 0.4), np.zeros((0, 6)))


def make_scene(w: Workload) -> Scene:
    g = rng(w.seed, STREAM_SCENE)
    if w.spacing > 0.0:
        cyl = poisson_disc_cylinders(g, w.n_cyl, w.r_in, w.r_out, w.rad_lo, w.rad_hi, w.spacing)
    else:
        cyl = annulus_cylinders(g, w.n_cyl, w.r_in, w.r_out, w.rad_lo, w.rad_hi)
    box = (annulus_boxes(g, w.n_box, w.box_r_in, w.box_r_out, w.box_side_lo, w.box_side_hi)
           if w.n_box else np.zeros((0, 6)))
    return Scene(cyl, box)


def uniform_configurations(model: CraneModel, g: np.random.Generator, n: int) -> np.ndarray:
    """n configurations uniform within the joint limits, float64 [n][4]."""
    lo = np.asarray(model.q_min)
    hi = np.asarray(model.q_max)
    return lo + (hi - lo) * g.random((n, 4))


def select_endpoints(model: CraneModel, distance: Callable[[np.ndarray], np.ndarray],
                     seed: int = 0, clearance: float = 1e-3, batch: int = 65536,
                     max_draws: int = 1_000_000, query: int = 0) -> tuple:
    """Start and goal: the first two draws (in draw order) of configurations uniform in the
    joint limits whose signed distance, as given by `distance`, exceeds `clearance`.

    The clearance keeps the choice away from grazing contact, where an FP32 and an FP64
    distance could disagree. When fewer than two draws qualify within `max_draws`, the
    least-penetrating draws are used and `ok` is False.
    Returns (q0, qd, ok, draws).
    """
    g = rng(seed, STREAM_ENDPOINTS, query)
    found: List[np.ndarray] = []
    best: List[tuple] = []
    draws = 0
    while draws < max_draws and len(found) < 2:
        q = uniform_configurations(model, g, batch)
        d = np.asarray(distance(q), dtype=np.float64)
        for i in np.nonzero(d > clearance)[0]:
            found.append(q[i])
            if len(found) == 2:
                break
        order = np.argsort(-d, kind="stable")[:2]
        best.extend((float(d[i]), q[i]) for i in order)
        draws += batch
    if len(found) == 2:
        return found[0], found[1], True, draws
    best.sort(key=lambda t: -t[0])
    return best[0][1], best[1][1], False, draws


# Grasp poses for the batched IK: the grapple centre of a collision-free configuration
# (clearance GRASP_CLEARANCE) at a height in GRASP_Z (logs on the ground and on a low pile),
# yaw equal to the slew angle, in the sparse single-query stand (20 trees).
IK_SCENE = "single_small"
GRASP_CLEARANCE = 0.05
GRASP_Z = (-0.5, 1.5)


def grasp_configurations(model: CraneModel, accept: Callable[[np.ndarray], np.ndarray], n: int,
                         seed: int = 0, batch: int = 65536, max_draws: int = 8_000_000) -> np.ndarray:
    """The first n draws (in draw order) of configurations uniform in the joint limits that
    `accept` admits; `accept` maps q[m][4] to bool[m] and is the caller's (the grasp rule
    above: distance and grapple height, evaluated by whichever implementation the caller
    trusts). float64 [n][4]; raises when fewer than n qualify within max_draws."""
    g = rng(seed, STREAM_IK_TARGETS)
    found: List[np.ndarray] = []
    have, draws = 0, 0
    while have < n and draws < max_draws:
        q = uniform_configurations(model, g, batch)
        ok = np.asarray(accept(q), dtype=bool)
        found.append(q[ok][: n - have])
        have += found[-1].shape[0]
        draws += batch
    if have < n:
        raise RuntimeError("only %d of %d grasp configurations in %d draws" % (have, n, draws))
    return np.concatenate(found, axis=0)


# --------------------------------------------------------------------------- test buffers

def straight_line_points(q0: np.ndarray, qd: np.ndarray, K: int) -> np.ndarray:
    """K points evenly spaced on the segment from q0 to qd (excluding both ends),
    float64 [K][4]. This is the data layout of an initial guess, not an evaluation."""
    f = (np.arange(1, K + 1, dtype=np.float64) / (K + 1))[:, None]
    return q0[None, :] + f * (qd - q0)[None, :]


def random_candidates(q0: np.ndarray, qd: np.ndarray, K: int, n: int, seed: int,
                      spread=(0.6, 0.3, 0.4, 0.5)) -> np.ndarray:
    """n candidate control-point sets around the straight line, float32 [n][K][4]."""
    g = rng(seed, STREAM_TEST, K, n)
    base = straight_line_points(np.asarray(q0, np.float64), np.asarray(qd, np.float64), K)
    noise = g.standard_normal((n, K, 4)) * np.asarray(spread)[None, None, :]
    return (base[None] + noise).astype(np.float32)


def random_costs(n: int, seed: int, ties: int = 0) -> np.ndarray:
    """n float64 costs (log-normal), with `ties` values repeated to exercise tie-breaking."""
    g = rng(seed, STREAM_TEST, 99, n)
    J = np.exp(g.standard_normal(n) * 2.0)
    if ties > 0 and n > 1:
        idx = g.integers(0, n, size=ties)
        J[idx] = J[idx[0]]
    return J

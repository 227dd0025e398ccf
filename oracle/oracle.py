"""FP64 CPU oracle of the stochastic B-spline path optimisation (arXiv 2503.14160, Sec. 4.1,
Algorithm 1) -- TEST INFRASTRUCTURE.

Only the test-suite, the package smoke check and the benchmark's CPU-baseline leg use
this module; the CUDA library never does, and the two share no code. The per-candidate
cost (kinematics, signed distances, Cox-de Boor spline, Eq. path opt) runs in the plain C
file next to this one; the steps of Algorithm 1 that act on the whole population are
written here with numpy, one function per step, in the paper's order and notation:

  init_distribution  initial mean mu (linear interpolation, evenly spaced interior
                     control points, Sec. 4.1) and initial covariance C
  factor             L with L L^T = sigma^2 C (numpy Cholesky), for step (1)
  sample             step (1): xi_i = mu + L z_i, z_i from Philox + Box-Muller
  sample_elites      step (1) from the last update's elites, no factor (same distribution)
  evaluate           step (2): J(xi_i) through the C oracle
  evaluate_grid      the same with d(q) through a uniform obstacle grid (timing only)
  rank               step (3): stable ascending sort of J (NaN sorts last)
  log_rank_weights   step (4): w_j = (ln(nu + 1/2) - ln j) / sum_k (ln(nu + 1/2) - ln k)
  update             steps (5) and (6): mu <- sum_j w_j x_(j);
                     C <- sum_j w_j (x_(j) - mu)(x_(j) - mu)^T + eps I  (new mu)
  plan               the loop of Algorithm 1 for a fixed number of iterations
  update_cmaes       the CMA-ES update the method is modelled on (step size and evolution
                     paths, rank-one and rank-mu covariance about the old mean), a variant
                     of steps (5) and (6)
  ik_residual        the residual of the collision-free IK (Sec. 3.2, Eq. IK opt) and its
                     Jacobian, through the C oracle
  ik_solve           damped Gauss-Newton (Levenberg-Marquardt) on Eq. IK opt from one start
  ik_solve_best      the best of several Philox starting points

Readings where the paper is silent: sigma = 1; C_0 = diag((0.1 (q_max - q_min))^2) per
free control point; nu = floor(N/2); eps = 1e-8; w_c = w_l = 100; lambda_c = 1; the
covariance uses the new mean; ties in the sort go to the lower candidate index.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import sys
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
if _HERE not in sys.path:
    sys.path.insert(0, _HERE)
import build as _build  # noqa: E402  (oracle/build.py)

O_MAX_SPHERES = 32


class _Model(ctypes.Structure):
    _fields_ = [("base_z", ctypes.c_double), ("boom_len", ctypes.c_double),
                ("jib_len", ctypes.c_double), ("q_min", ctypes.c_double * 4),
                ("q_max", ctypes.c_double * 4), ("n_spheres", ctypes.c_int32),
                ("link", ctypes.c_int32 * O_MAX_SPHERES),
                ("offset", ctypes.c_double * O_MAX_SPHERES),
                ("radius", ctypes.c_double * O_MAX_SPHERES)]


class _Scene(ctypes.Structure):
    _fields_ = [("n_cyl", ctypes.c_int32), ("cyl", ctypes.POINTER(ctypes.c_double)),
                ("n_box", ctypes.c_int32), ("box", ctypes.POINTER(ctypes.c_double))]


class _CostParams(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("S", ctypes.c_int32), ("w_c", ctypes.c_double),
                ("w_l", ctypes.c_double), ("lambda_c", ctypes.c_double),
                ("margin", ctypes.c_double), ("beta", ctypes.c_double)]


class _Cost(ctypes.Structure):
    _fields_ = [("J", ctypes.c_double), ("Jp", ctypes.c_double), ("Jc", ctypes.c_double),
                ("Jl", ctypes.c_double), ("length", ctypes.c_double),
                ("flag", ctypes.c_int32), ("n_flagged", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.o_philox4x32_10_batch.argtypes = [u32p, u32p, ctypes.c_int64, u32p]
        L.o_normals_batch.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_int32, ctypes.c_int32, dp]
        L.o_fk.argtypes = [ctypes.POINTER(_Model), dp, dp, dp, dp]
        L.o_fk_tip_batch.argtypes = [ctypes.POINTER(_Model), dp, ctypes.c_int64, dp]
        L.o_sdf_cylinder.argtypes = [dp, dp]
        L.o_sdf_cylinder.restype = ctypes.c_double
        L.o_sdf_box.argtypes = [dp, dp]
        L.o_sdf_box.restype = ctypes.c_double
        L.o_signed_distance_batch.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Scene),
                                              dp, ctypes.c_int64, dp]
        L.o_bspline_basis.argtypes = [ctypes.c_int32, ctypes.c_double, dp]
        L.o_bspline.argtypes = [dp, ctypes.c_int32, ctypes.c_double, dp]
        L.o_path_cost_batch.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Scene),
                                        ctypes.POINTER(_CostParams), dp, ctypes.c_int64,
                                        dp, dp, ctypes.POINTER(_Cost), dp]
        L.o_path_cost_batch_grid.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Scene),
                                             ctypes.POINTER(_CostParams), dp, ctypes.c_int64,
                                             dp, dp, ctypes.c_double, ctypes.POINTER(_Cost), dp]
        L.o_path_cost_batch_grid.restype = ctypes.c_int32
        L.o_smooth_cost_batch.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Scene),
                                          ctypes.POINTER(_CostParams), dp, ctypes.c_int64,
                                          dp, dp, dp]
        L.o_smooth_grad_batch.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Scene),
                                          ctypes.POINTER(_CostParams), dp, ctypes.c_int64,
                                          dp, dp, dp]
        L.o_ik_residual.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Scene), dp, dp,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
        L.o_set_threads.argtypes = [ctypes.c_int32]
        L.o_get_threads.restype = ctypes.c_int32
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().o_set_threads(int(n))


def get_threads() -> int:
    return int(lib().o_get_threads())


# --------------------------------------------------------------------------- inputs

@dataclasses.dataclass
class CostParams:
    K: int
    S: int
    w_c: float = 100.0
    w_l: float = 100.0
    lambda_c: float = 1.0
    margin: float = 0.05
    beta: float = 0.01

    @property
    def n_checkpoints(self) -> int:
        return (self.K + 3) * self.S


class Problem:
    """The crane model, the obstacle scene and the cost weights in the C oracle's layout."""

    def __init__(self, model, scene, cost: CostParams):
        self.model_py = model
        m = _Model()
        m.base_z, m.boom_len, m.jib_len = model.base_z, model.boom_len, model.jib_len
        for c in range(4):
            m.q_min[c], m.q_max[c] = model.q_min[c], model.q_max[c]
        if len(model.spheres) > O_MAX_SPHERES:
            raise ValueError("too many spheres")
        m.n_spheres = len(model.spheres)
        for s, sp in enumerate(model.spheres):
            m.link[s], m.offset[s], m.radius[s] = sp.link, sp.offset, sp.radius
        self.model = m
        self.cyl = _c64(scene.cylinders).reshape(-1, 5)
        self.box = _c64(scene.boxes).reshape(-1, 6)
        sc = _Scene()
        sc.n_cyl, sc.cyl = self.cyl.shape[0], _dp(self.cyl)
        sc.n_box, sc.box = self.box.shape[0], _dp(self.box)
        self.scene = sc
        if cost.K + 8 > 64:
            raise ValueError("the oracle supports at most 56 waypoints")
        self.cost = cost
        self.cp = _CostParams(cost.K, cost.S, cost.w_c, cost.w_l, cost.lambda_c,
                              cost.margin, cost.beta)


# --------------------------------------------------------------------------- primitives

def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of counters ctr[n][4] (uint32) under key (k0, k1)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros_like(ctr)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().o_philox4x32_10_batch(ctr.ctypes.data_as(u32p), k.ctypes.data_as(u32p),
                                ctr.shape[0], out.ctypes.data_as(u32p))
    return out


def normals(seed: int, t: int, query: int, n: int, K: int) -> np.ndarray:
    """z[n][4K]: the standard normals of candidates 0..n-1 at iteration t."""
    z = np.zeros((n, 4 * K))
    lib().o_normals_batch(seed, t, query, n, K, _dp(z))
    return z


def fk(problem: Problem, q) -> tuple:
    """(centres[n_spheres][3], jib pivot J[3], tip T[3]) at configuration q."""
    q = _c64(q).reshape(4)
    n = problem.model.n_spheres
    c = np.zeros((n, 3))
    J = np.zeros(3)
    T = np.zeros(3)
    lib().o_fk(ctypes.byref(problem.model), _dp(q), _dp(c), _dp(J), _dp(T))
    return c, J, T


def fk_tips(problem: Problem, q) -> np.ndarray:
    """Tips T[n][3] of configurations q[n][4] (the T of fk, batched)."""
    q = _c64(q).reshape(-1, 4)
    T = np.zeros((q.shape[0], 3))
    lib().o_fk_tip_batch(ctypes.byref(problem.model), _dp(q), q.shape[0], _dp(T))
    return T


def sdf_cylinder(p, cyl) -> float:
    return float(lib().o_sdf_cylinder(_dp(_c64(p)), _dp(_c64(cyl))))


def sdf_box(p, box) -> float:
    return float(lib().o_sdf_box(_dp(_c64(p)), _dp(_c64(box))))


def signed_distance(problem: Problem, q) -> np.ndarray:
    """d(q) for configurations q[n][4] (Sec. 3.1; d < 0 is collision)."""
    q = _c64(q).reshape(-1, 4)
    d = np.zeros(q.shape[0])
    lib().o_signed_distance_batch(ctypes.byref(problem.model), ctypes.byref(problem.scene),
                                  _dp(q), q.shape[0], _dp(d))
    return d


def bspline_basis(n_c: int, tau: float) -> np.ndarray:
    b = np.zeros(n_c)
    lib().o_bspline_basis(n_c, float(tau), _dp(b))
    return b


def bspline(P, tau: float) -> np.ndarray:
    P = _c64(P).reshape(-1, 4)
    q = np.zeros(4)
    lib().o_bspline(_dp(P), P.shape[0], float(tau), _dp(q))
    return q


@dataclasses.dataclass
class Costs:
    J: np.ndarray
    Jp: np.ndarray
    Jc: np.ndarray
    Jl: np.ndarray
    length: np.ndarray
    flag: np.ndarray
    n_flagged: np.ndarray
    d: Optional[np.ndarray] = None   # [n][n_s + 1] signed distance at every checkpoint


def evaluate(problem: Problem, xi, q0, qd, with_distances: bool = False) -> Costs:
    """Algorithm 1 step (2): the cost of Eq. path opt for candidates xi[n][K][4]."""
    K = problem.cost.K
    xi = _c64(xi).reshape(-1, K, 4)
    n = xi.shape[0]
    out = (_Cost * max(n, 1))()
    d = np.zeros((n, problem.cost.n_checkpoints + 1)) if with_distances else None
    lib().o_path_cost_batch(ctypes.byref(problem.model), ctypes.byref(problem.scene),
                            ctypes.byref(problem.cp), _dp(xi), n, _dp(_c64(q0)), _dp(_c64(qd)),
                            out, _dp(d) if d is not None else None)
    arr = np.ctypeslib.as_array(out)[:n]
    return Costs(arr["J"].copy(), arr["Jp"].copy(), arr["Jc"].copy(), arr["Jl"].copy(),
                 arr["length"].copy(), arr["flag"].copy(), arr["n_flagged"].copy(), d)


def evaluate_grid(problem: Problem, xi, q0, qd, cell: float, with_distances: bool = False) -> Costs:
    """evaluate() with d(q) through a uniform obstacle grid of cell side `cell` (m): the same
    costs and flags as the brute force (only negative distances enter them), much faster on
    large scenes. For timing the oracle on the dense forest; the parity tests use evaluate()."""
    K = problem.cost.K
    xi = _c64(xi).reshape(-1, K, 4)
    n = xi.shape[0]
    out = (_Cost * max(n, 1))()
    d = np.zeros((n, problem.cost.n_checkpoints + 1)) if with_distances else None
    rc = lib().o_path_cost_batch_grid(ctypes.byref(problem.model), ctypes.byref(problem.scene),
                                      ctypes.byref(problem.cp), _dp(xi), n, _dp(_c64(q0)), _dp(_c64(qd)),
                                      ctypes.c_double(cell), out, _dp(d) if d is not None else None)
    if rc != 0:
        raise MemoryError("oracle grid of cell %g could not be built" % cell)
    arr = np.ctypeslib.as_array(out)[:n]
    return Costs(arr["J"].copy(), arr["Jp"].copy(), arr["Jc"].copy(), arr["Jl"].copy(),
                 arr["length"].copy(), arr["flag"].copy(), arr["n_flagged"].copy(), d)


def smooth_cost(problem: Problem, xi, q0, qd) -> np.ndarray:
    """The cost with the softplus collision penalty, for candidates xi[n][K][4]."""
    K = problem.cost.K
    xi = _c64(xi).reshape(-1, K, 4)
    J = np.zeros(xi.shape[0])
    lib().o_smooth_cost_batch(ctypes.byref(problem.model), ctypes.byref(problem.scene),
                              ctypes.byref(problem.cp), _dp(xi), xi.shape[0], _dp(_c64(q0)),
                              _dp(_c64(qd)), _dp(J))
    return J


def smooth_grad(problem: Problem, xi, q0, qd) -> np.ndarray:
    """Analytic gradient of smooth_cost with respect to xi[n][K][4]."""
    K = problem.cost.K
    xi = _c64(xi).reshape(-1, K, 4)
    g = np.zeros_like(xi)
    lib().o_smooth_grad_batch(ctypes.byref(problem.model), ctypes.byref(problem.scene),
                              ctypes.byref(problem.cp), _dp(xi), xi.shape[0], _dp(_c64(q0)),
                              _dp(_c64(qd)), _dp(g))
    return g


def polish(problem: Problem, xi, q0, qd, steps: int, alpha: float) -> np.ndarray:
    """Plain gradient descent on the smooth cost, xi <- xi - alpha grad, `steps` times."""
    x = _c64(xi).reshape(-1, problem.cost.K, 4).copy()
    for _ in range(steps):
        x = x - alpha * smooth_grad(problem, x, q0, qd)
    return x


# --------------------------------------------------------------------------- Algorithm 1

@dataclasses.dataclass
class SearchParams:
    N: int
    K: int
    S: int
    nu: int = 0                 # 0: floor(N / 2)
    sigma: float = 1.0
    eps: float = 1e-8
    init_std_frac: float = 0.1
    seed: int = 0
    query: int = 0

    @property
    def n_elites(self) -> int:
        return self.nu if self.nu > 0 else self.N // 2


def init_distribution(q0, qd, K: int, q_min, q_max, init_std_frac: float = 0.1):
    """Initial mean: the K interior control points evenly spaced on the segment q0 -> qd
    (P_{3+i} = q0 + i/(K+1) (qd - q0), i = 1..K); initial covariance: diagonal, per joint
    (init_std_frac * (q_max - q_min))^2. Both flattened to D = 4K (point-major)."""
    q0, qd = _c64(q0), _c64(qd)
    i = np.arange(1, K + 1, dtype=np.float64)[:, None]
    mu = (q0[None, :] + i / (K + 1) * (qd - q0)[None, :]).reshape(-1)
    std = init_std_frac * (_c64(q_max) - _c64(q_min))
    C = np.diag(np.tile(std * std, K))
    return mu, C


def factor(C: np.ndarray, sigma: float) -> np.ndarray:
    """Lower-triangular L with L L^T = sigma^2 C."""
    return np.linalg.cholesky(sigma * sigma * C)


def sample(mu: np.ndarray, L: np.ndarray, seed: int, t: int, query: int, N: int, K: int):
    """Step (1): xi_i = mu + L z_i ~ N(mu, sigma^2 C), i = 0..N-1; returns [N][K][4]."""
    z = normals(seed, t, query, N, K)
    return (mu[None, :] + z @ L.T).reshape(N, K, 4)


def sample_elites(mu: np.ndarray, elites: np.ndarray, w: np.ndarray, sigma: float, eps: float,
                  seed: int, t: int, query: int, N: int, K: int):
    """Step (1) drawn from the elites of the last update, with no factor. With
    C = sum_j w_j (x_(j) - mu)(x_(j) - mu)^T + eps I (steps (5)-(6), mu the new mean),
        xi_i = mu + sigma (sum_j sqrt(w_j) (x_(j) - mu) g_ij + sqrt(eps) g'_i)
    is normal with mean mu and covariance sigma^2 C exactly. g_i are the first nu standard
    normals of candidate i's Philox stream at iteration t (blocks of four as in `normals`),
    g'_i the next D. Returns [N][K][4]."""
    D = 4 * K
    nu = len(w)
    X = _c64(elites).reshape(nu, D)
    z = normals(seed, t, query, N, (nu + D + 3) // 4)
    Y = np.sqrt(_c64(w))[:, None] * (X - _c64(mu)[None, :])
    xi = _c64(mu)[None, :] + sigma * (z[:, :nu] @ Y + math.sqrt(eps) * z[:, nu:nu + D])
    return xi.reshape(N, K, 4)


def rank(J: np.ndarray) -> np.ndarray:
    """Step (3): candidate indices in ascending order of J; stable (ties keep the lower
    index first); NaN costs sort after every number."""
    key = np.where(np.isnan(J), np.inf, J)
    return np.argsort(key, kind="stable")


def log_rank_weights(nu: int) -> np.ndarray:
    """Step (4): w_j = (ln(nu + 0.5) - ln j) / sum_{k=1}^{nu} (ln(nu + 0.5) - ln k)."""
    j = np.arange(1, nu + 1, dtype=np.float64)
    raw = math.log(nu + 0.5) - np.log(j)
    return raw / raw.sum()


def update(xi: np.ndarray, J: np.ndarray, nu: int, eps: float):
    """Steps (3)-(6): select the nu elites, weight them by rank, and return the new mean
    and covariance (covariance about the new mean, plus eps I)."""
    D = xi.shape[1] * xi.shape[2] if xi.ndim == 3 else xi.shape[1]
    X = _c64(xi).reshape(-1, D)
    order = rank(J)
    elites = X[order[:nu]]
    w = log_rank_weights(nu)
    mu = w @ elites
    Y = elites - mu[None, :]
    C = (Y * w[:, None]).T @ Y + eps * np.eye(D)
    return mu, C


# --------------------------------------------------------------------------- CMA-ES variant

@dataclasses.dataclass
class CMAState:
    """State of the CMA-ES update (the variant the paper's method is modelled on): mean,
    covariance, global step size sigma, the two evolution paths, and the iterations done."""
    mu: np.ndarray
    C: np.ndarray
    sigma: float
    p_sigma: np.ndarray
    p_c: np.ndarray
    t: int = 0


@dataclasses.dataclass
class CMAConstants:
    mu_eff: float
    c_sigma: float
    d_sigma: float
    c_c: float
    c_1: float
    c_mu: float
    chi_n: float


def cma_constants(D: int, w: np.ndarray) -> CMAConstants:
    """Default learning rates of CMA-ES for dimension D and positive recombination weights
    w (Hansen, "The CMA Evolution Strategy: A Tutorial", 2016, Table 1), and the expected
    norm of a D-dimensional standard normal vector (its series approximation)."""
    mu_eff = 1.0 / float(np.sum(w * w))
    c_sigma = (mu_eff + 2.0) / (D + mu_eff + 5.0)
    d_sigma = 1.0 + 2.0 * max(0.0, math.sqrt((mu_eff - 1.0) / (D + 1.0)) - 1.0) + c_sigma
    c_c = (4.0 + mu_eff / D) / (D + 4.0 + 2.0 * mu_eff / D)
    c_1 = 2.0 / ((D + 1.3) ** 2 + mu_eff)
    c_mu = min(1.0 - c_1, 2.0 * (mu_eff - 2.0 + 1.0 / mu_eff) / ((D + 2.0) ** 2 + mu_eff))
    chi_n = math.sqrt(D) * (1.0 - 1.0 / (4.0 * D) + 1.0 / (21.0 * D * D))
    return CMAConstants(mu_eff, c_sigma, d_sigma, c_c, c_1, c_mu, chi_n)


def cma_init(mu: np.ndarray, C: np.ndarray, sigma: float) -> CMAState:
    D = mu.shape[0]
    return CMAState(_c64(mu).copy(), _c64(C).copy(), float(sigma), np.zeros(D), np.zeros(D), 0)


def update_cmaes(state: CMAState, xi: np.ndarray, J: np.ndarray, nu: int) -> CMAState:
    """CMA-ES update in place of steps (5) and (6), with the same selection and weights
    (steps (3) and (4)), in the order of the tutorial:
      mean      m' = sum_j w_j x_(j)
      steps     y_j = (x_(j) - m) / sigma          (about the OLD mean)
      p_sigma   (1 - c_s) p_sigma + sqrt(c_s (2 - c_s) mu_eff) L_C^-1 (m' - m) / sigma
      h_sigma   1 if |p_sigma| / sqrt(1 - (1 - c_s)^(2 (t + 1))) < (1.4 + 2 / (D + 1)) chi_n
      p_c       (1 - c_c) p_c + h_sigma sqrt(c_c (2 - c_c) mu_eff) (m' - m) / sigma
      C'        (1 + c_1 (1 - h_sigma) c_c (2 - c_c) - c_1 - c_mu) C + c_1 p_c p_c^T
                + c_mu sum_j w_j y_j y_j^T
      sigma'    sigma exp((c_s / d_s) (|p_sigma| / chi_n - 1))
    C^-1/2 of the tutorial is taken as L_C^-1 with L_C the Cholesky factor of C: both map
    N(0, C) to N(0, I), which is all the path's length statistics rely on."""
    D = state.mu.shape[0]
    X = _c64(xi).reshape(-1, D)
    order = rank(J)
    elites = X[order[:nu]]
    w = log_rank_weights(nu)
    k = cma_constants(D, w)
    m, sigma = state.mu, state.sigma
    m_new = w @ elites
    Y = (elites - m[None, :]) / sigma
    L_C = np.linalg.cholesky(state.C)
    shift = (m_new - m) / sigma
    z = np.linalg.solve(L_C, shift)
    p_sigma = (1.0 - k.c_sigma) * state.p_sigma + math.sqrt(k.c_sigma * (2.0 - k.c_sigma) * k.mu_eff) * z
    norm = float(np.linalg.norm(p_sigma))
    h = 1.0 if norm / math.sqrt(1.0 - (1.0 - k.c_sigma) ** (2 * (state.t + 1))) < (1.4 + 2.0 / (D + 1)) * k.chi_n else 0.0
    p_c = (1.0 - k.c_c) * state.p_c + h * math.sqrt(k.c_c * (2.0 - k.c_c) * k.mu_eff) * shift
    delta_h = (1.0 - h) * k.c_c * (2.0 - k.c_c)
    C = ((1.0 + k.c_1 * delta_h - k.c_1 - k.c_mu) * state.C + k.c_1 * np.outer(p_c, p_c)
         + k.c_mu * (Y * w[:, None]).T @ Y)
    sigma_new = sigma * math.exp((k.c_sigma / k.d_sigma) * (norm / k.chi_n - 1.0))
    return CMAState(m_new, C, sigma_new, p_sigma, p_c, state.t + 1)


@dataclasses.dataclass
class PlanResult:
    mu: np.ndarray              # final mean, [K][4]
    C: np.ndarray               # final covariance
    control_points: np.ndarray  # [K+8][4], end copies included
    best_J: np.ndarray          # per iteration: min over the population
    mean_J: np.ndarray          # per iteration: cost of the mean path after the update
    final: Costs                # cost terms of the final mean path


def plan(problem: Problem, sp: SearchParams, q0, qd, iterations: int,
         callback=None, rule: str = "paper", sampler: str = "factor",
         cost_noise: Optional[tuple] = None) -> PlanResult:
    """Algorithm 1 for a fixed number of iterations, starting from init_distribution;
    rule "cmaes" takes update_cmaes (sigma adapted) in place of steps (5)-(6); sampler
    "elites" (paper rule) draws every sample after the first with sample_elites.
    cost_noise = (rel, seed), for sensitivity studies only: every cost the ranking sees is
    multiplied by (1 + rel g), g standard normal from numpy's generator under `seed`, which
    stands for evaluation errors of relative size rel (None: exact FP64 costs)."""
    q0, qd = _c64(q0), _c64(qd)
    m = problem.model_py
    mu, C = init_distribution(q0, qd, sp.K, m.q_min, m.q_max, sp.init_std_frac)
    st = cma_init(mu, C, sp.sigma)
    best, mean_J = [], []
    last = None   # (mean, elites in rank order, weights) of the last paper-rule update
    for t in range(iterations):
        if sampler == "elites" and last is not None:
            xi = sample_elites(last[0], last[1], last[2], sp.sigma, sp.eps, sp.seed, t, sp.query, sp.N, sp.K)
        else:
            L = factor(st.C if rule == "cmaes" else C, st.sigma if rule == "cmaes" else sp.sigma)
            xi = sample(st.mu if rule == "cmaes" else mu, L, sp.seed, t, sp.query, sp.N, sp.K)
        J = evaluate(problem, xi, q0, qd).J
        if cost_noise is not None:
            if t == 0:
                noise = np.random.default_rng(cost_noise[1])
            J = J * (1.0 + cost_noise[0] * noise.standard_normal(J.shape))
        if rule == "cmaes":
            st = update_cmaes(st, xi, J, sp.n_elites)
            mu, C = st.mu, st.C
        else:
            mu, C = update(xi, J, sp.n_elites, sp.eps)
            X = _c64(xi).reshape(sp.N, -1)
            last = (mu, X[rank(J)[:sp.n_elites]], log_rank_weights(sp.n_elites))
        best.append(float(np.nanmin(J)))
        if callback is not None:
            callback(t, mu, C, J)
    final = evaluate(problem, mu.reshape(1, sp.K, 4), q0, qd)
    mean_J.append(float(final.J[0]))
    P = np.concatenate([np.tile(q0, (4, 1)), mu.reshape(sp.K, 4), np.tile(qd, (4, 1))])
    return PlanResult(mu.reshape(sp.K, 4), C, P, np.asarray(best), np.asarray(mean_J), final)


# --------------------------------------------------------------------------- collision-free IK

@dataclasses.dataclass
class IKParams:
    """Scales of the residual of Eq. IK opt (Sec. 3.2) and the solver's settings."""
    lambda_q: float = 1.0       # m per rad of yaw error
    lambda_c: float = 1.0       # scale of r_c = lambda_c max(0, -d)
    grapple_len: float = 1.0    # the grapple centre hangs this far below the tip (m)
    mu0: float = 1e-3           # initial damping
    seed: int = 0               # Philox key of the starting points


IK_TAG = 0x494B5354             # third Philox counter word of the IK starting points


def ik_residual(problem: Problem, q, target, ik: IKParams, jacobian: bool = True):
    """r (5) and, if asked, dr/dq (5 x 4) of Eq. IK opt at q for target (x, y, z, psi)."""
    r = np.zeros(5)
    J = np.zeros((5, 4)) if jacobian else None
    lib().o_ik_residual(ctypes.byref(problem.model), ctypes.byref(problem.scene), _dp(_c64(q)),
                        _dp(_c64(target)), ik.lambda_q, ik.lambda_c, ik.grapple_len, _dp(r),
                        _dp(J) if J is not None else None)
    return r, J


def ik_start(problem: Problem, ik: IKParams, target_index: int, restart: int, query: int = 0):
    """Starting configuration `restart` of target `target_index`: four uniforms from one
    Philox4x32-10 block (counter (restart, target, tag, query), key = seed), top 24 bits of
    each word, spread over the joint limits."""
    ctr = np.array([[restart, target_index, IK_TAG, query]], dtype=np.uint32)
    key = (int(ik.seed) & 0xFFFFFFFF, (int(ik.seed) >> 32) & 0xFFFFFFFF)
    w = philox4x32_10(ctr, key)[0]
    u = (w >> 8).astype(np.float64) * 2.0 ** -24
    lo = np.array(problem.model_py.q_min, dtype=np.float64)
    hi = np.array(problem.model_py.q_max, dtype=np.float64)
    return lo + u * (hi - lo)


def ik_solve(problem: Problem, target, q_start, iters: int, ik: IKParams):
    """Damped Gauss-Newton (Levenberg-Marquardt) on Eq. IK opt from q_start, the steps in
    order: H = J^T J, g = J^T r; solve (H + mu (diag H + 1e-6)) s = -g; q' = clip(q + s)
    to the joint limits; accept q' when |r(q')|^2 < |r(q)|^2 (then mu /= 3, floor 1e-12),
    else mu *= 4 (cap 1e12). Returns (q, |r|^2, history of |r|^2 after each iteration)."""
    lo = np.array(problem.model_py.q_min, dtype=np.float64)
    hi = np.array(problem.model_py.q_max, dtype=np.float64)
    q = np.clip(_c64(q_start), lo, hi)
    mu = ik.mu0
    r, J = ik_residual(problem, q, target, ik)
    f = float(r @ r)
    hist = []
    for _ in range(iters):
        H = J.T @ J
        g = J.T @ r
        A = H + mu * np.diag(np.diag(H) + 1e-6)
        step = -np.linalg.solve(A, g)
        q_new = np.clip(q + step, lo, hi)
        r_new, J_new = ik_residual(problem, q_new, target, ik)
        f_new = float(r_new @ r_new)
        if f_new < f:
            q, r, J, f = q_new, r_new, J_new, f_new
            mu = max(mu / 3.0, 1e-12)
        else:
            mu = min(mu * 4.0, 1e12)
        hist.append(f)
    return q, f, hist


def ik_solve_best(problem: Problem, target, target_index: int, restarts: int, iters: int,
                  ik: IKParams, query: int = 0):
    """The best of `restarts` solves from the Philox starting points (lowest |r|^2, ties to
    the lower restart index): (q, |r|^2, restart)."""
    best = None
    for s in range(restarts):
        q, f, _ = ik_solve(problem, target, ik_start(problem, ik, target_index, s, query), iters, ik)
        if best is None or f < best[1]:
            best = (q, f, s)
    return best

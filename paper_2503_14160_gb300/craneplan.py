"""Python binding of the craneplan C ABI (include/craneplan.h): argument marshalling only.

Every function keeps the name of the C entry point it calls. Device buffers are passed as
torch CUDA tensors (their data pointers); host buffers as numpy arrays or sequences. The
CUDA library must have been built (``paper_2503_14160_gb300.build.build()``); there is no
fallback: importing this module without the library raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

CP_MAX_SPHERES = 16
CP_MAX_WAYPOINTS = 32

STATUS = {0: "CP_OK", -1: "CP_ERR_ARG", -2: "CP_ERR_CUDA", -3: "CP_ERR_TIMEOUT",
          -4: "CP_ERR_STATE", -5: "CP_ERR_OOM", -6: "CP_ERR_NUMERIC"}


class CranePlanError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class cp_sphere(ctypes.Structure):
    _fields_ = [("link", ctypes.c_int32), ("offset", ctypes.c_double), ("radius", ctypes.c_double)]


class cp_model(ctypes.Structure):
    _fields_ = [("base_z", ctypes.c_double), ("boom_len", ctypes.c_double),
                ("jib_len", ctypes.c_double), ("q_min", ctypes.c_double * 4),
                ("q_max", ctypes.c_double * 4), ("n_spheres", ctypes.c_int32),
                ("spheres", cp_sphere * CP_MAX_SPHERES)]


class cp_cylinder(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("radius", ctypes.c_double),
                ("z_lo", ctypes.c_double), ("z_hi", ctypes.c_double)]


class cp_box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class cp_scene(ctypes.Structure):
    _fields_ = [("n_cyl", ctypes.c_int32), ("cyl", ctypes.c_void_p),
                ("n_box", ctypes.c_int32), ("box", ctypes.c_void_p)]


class cp_params(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int32), ("n_waypoints", ctypes.c_int32),
                ("substeps", ctypes.c_int32), ("n_elites", ctypes.c_int32),
                ("w_c", ctypes.c_double), ("w_l", ctypes.c_double),
                ("lambda_c", ctypes.c_double), ("sigma", ctypes.c_double),
                ("eps", ctypes.c_double), ("init_std_frac", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("query", ctypes.c_uint32),
                ("max_cylinders", ctypes.c_int32), ("max_boxes", ctypes.c_int32),
                ("grid_cell", ctypes.c_double), ("grid_half_extent", ctypes.c_double),
                ("max_grid_items", ctypes.c_int64), ("smooth_margin", ctypes.c_double),
                ("smooth_beta", ctypes.c_double), ("eval_ctas_per_sm", ctypes.c_int32),
                ("debug_withhold_staging", ctypes.c_int32), ("eval_exhaustive", ctypes.c_int32),
                ("update_rule", ctypes.c_int32), ("collision_model", ctypes.c_int32),
                ("sampler", ctypes.c_int32)]


CP_UPDATE_PAPER = 0
CP_UPDATE_CMAES = 1
CP_SAMPLE_FACTOR = 0
CP_SAMPLE_ELITES = 1
CP_COLLISION_SPHERES = 0
CP_COLLISION_HULLS = 1


class cp_plan_stats(ctypes.Structure):
    _fields_ = [("J", ctypes.c_double), ("Jp", ctypes.c_double), ("Jc", ctypes.c_double),
                ("Jl", ctypes.c_double), ("length", ctypes.c_double),
                ("flag", ctypes.c_int32), ("n_flagged", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("iteration", ctypes.c_int32),
                ("best_J", ctypes.c_double)]


class cp_query(ctypes.Structure):
    _fields_ = [("scene", cp_scene), ("params", cp_params), ("q0", ctypes.c_double * 4),
                ("qd", ctypes.c_double * 4)]


class cp_batch_shape(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("items_per_warp", ctypes.c_int32)]


class cp_batch_info(ctypes.Structure):
    _fields_ = [("kernel_nodes", ctypes.c_int64), ("eval_tiles", ctypes.c_int64),
                ("eval_ctas", ctypes.c_int32), ("eval_launches", ctypes.c_int32),
                ("candidates", ctypes.c_int64), ("last_run_ms", ctypes.c_double)]


class cp_batch_result(ctypes.Structure):
    _fields_ = [("stats", cp_plan_stats), ("ctrl", ctypes.c_double * ((CP_MAX_WAYPOINTS + 8) * 4))]


class cp_timing(ctypes.Structure):
    _fields_ = [("eval_ms", ctypes.c_double), ("eval_launches", ctypes.c_int64),
                ("sample_ms", ctypes.c_double), ("sample_launches", ctypes.c_int64),
                ("factor_ms", ctypes.c_double), ("factor_launches", ctypes.c_int64),
                ("update_ms", ctypes.c_double), ("update_launches", ctypes.c_int64),
                ("eval_units", ctypes.c_int64), ("eval_obstacle_tests", ctypes.c_int64),
                ("eval_pair_tests", ctypes.c_int64), ("eval_box_tests", ctypes.c_int64)]


class cp_hull_model(ctypes.Structure):
    _fields_ = [("w", ctypes.c_double * 3), ("h", ctypes.c_double * 3), ("pad", ctypes.c_double),
                ("grapple_w", ctypes.c_double), ("grapple_len", ctypes.c_double)]


class cp_traj_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("omega_s", ctypes.c_double), ("omega_t", ctypes.c_double),
                ("R", ctypes.c_double * 4), ("dq_max", ctypes.c_double * 4), ("swing_max", ctypes.c_double),
                ("grapple_len", ctypes.c_double), ("rho", ctypes.c_double), ("rho_b", ctypes.c_double),
                ("outer", ctypes.c_int32), ("inner", ctypes.c_int32), ("mu0", ctypes.c_double)]


def make_traj_params(N: int = 100, omega_s: float = 1e-2, omega_t: float = 1e2, R=(1.0, 1.0, 1.0, 1.0),
                     dq_max=(0.6, 0.3, 0.3, 0.5), swing_max: float = 0.6, grapple_len: float = 1.0,
                     rho: float = 3e3, rho_b: float = 1e5, outer: int = 12, inner: int = 10,
                     mu0: float = 1e-3) -> "cp_traj_params":
    return cp_traj_params(int(N), float(omega_s), float(omega_t), (ctypes.c_double * 4)(*R),
                          (ctypes.c_double * 4)(*dq_max), float(swing_max), float(grapple_len), float(rho),
                          float(rho_b), int(outer), int(inner), float(mu0))


class cp_ik_params(ctypes.Structure):
    _fields_ = [("lambda_q", ctypes.c_double), ("lambda_c", ctypes.c_double),
                ("grapple_len", ctypes.c_double), ("mu0", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("query", ctypes.c_uint32),
                ("restarts", ctypes.c_int32), ("iters", ctypes.c_int32)]


CP_IK_MAX_RESTARTS = 1024

_P = ctypes.c_void_p
_SIGS = {
    "cp_last_error": (ctypes.c_char_p, []),
    "cp_version": (ctypes.c_int32, []),
    "cp_launch_count": (ctypes.c_int64, []),
    "cp_debug_fail_allocations": (None, [ctypes.c_int32]),
    "cp_debug_static_withhold_staging": (None, [ctypes.c_int32]),
    "cp_plan_init": (ctypes.c_int, [ctypes.POINTER(cp_model), ctypes.POINTER(cp_scene),
                                    ctypes.POINTER(cp_params), _P, ctypes.POINTER(_P)]),
    "cp_destroy": (None, [_P]),
    "cp_set_scene": (ctypes.c_int, [_P, ctypes.POINTER(cp_scene)]),
    "cp_set_endpoints": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
    "cp_sample": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "cp_evaluate": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, _P, _P, _P]),
    "cp_update": (ctypes.c_int, [_P, _P, _P]),
    "cp_synchronize": (ctypes.c_int, [_P]),
    "cp_plan": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(cp_plan_stats)]),
    "cp_signed_distance": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
    "cp_forward_kinematics": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
    "cp_hull_penetration": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(cp_hull_model), _P]),
    "cp_set_hull_model": (ctypes.c_int, [_P, ctypes.POINTER(cp_hull_model)]),
    "cp_ik": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(cp_ik_params), _P, _P, _P,
                             _P, _P]),
    "cp_get_distribution": (ctypes.c_int, [_P, _P, _P]),
    "cp_set_distribution": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
    "cp_get_factor": (ctypes.c_int, [_P, _P]),
    "cp_get_cma_state": (ctypes.c_int, [_P, _P]),
    "cp_set_cma_state": (ctypes.c_int, [_P, _P]),
    "cp_get_elites": (ctypes.c_int, [_P, _P]),
    "cp_get_population": (ctypes.c_int, [_P, _P, _P]),
    "cp_set_metrics": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cp_get_metrics": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32)]),
    "cp_philox4x32_10": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64, _P, _P]),
    "cp_evaluate_static": (ctypes.c_int, [ctypes.POINTER(cp_model), _P, ctypes.c_int32, _P,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), _P, ctypes.c_int32,
                                          _P, _P, _P, _P]),
    "cp_smooth_cost": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
    "cp_smooth_cost_grad": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, _P]),
    "cp_polish": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double]),
    "cp_batch_init": (ctypes.c_int, [ctypes.POINTER(cp_model), ctypes.POINTER(cp_query),
                                     ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)]),
    "cp_batch_set_endpoints": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]),
    "cp_batch_run": (ctypes.c_int, [_P, ctypes.POINTER(cp_batch_result)]),
    "cp_batch_planner": (_P, [_P, ctypes.c_int32]),
    "cp_batch_set_shape": (ctypes.c_int, [_P, ctypes.POINTER(cp_batch_shape)]),
    "cp_batch_evaluate": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "cp_batch_get_info": (ctypes.c_int, [_P, ctypes.POINTER(cp_batch_info)]),
    "cp_batch_destroy": (None, [_P]),
    "cp_set_timing": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cp_get_timing": (ctypes.c_int, [_P, ctypes.POINTER(cp_timing)]),
    "cp_alu_peaks": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "cp_traj_init": (ctypes.c_int, [ctypes.POINTER(cp_model), ctypes.POINTER(cp_traj_params), ctypes.c_int32, _P,
                                    ctypes.POINTER(_P)]),
    "cp_traj_destroy": (None, [_P]),
    "cp_traj_targets": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "cp_traj_initial_guess": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
    "cp_traj_step": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, ctypes.c_double, _P]),
    "cp_traj_solve": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libcraneplan.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libcraneplan.so is not built (%s); run "
                           "paper_2503_14160_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise CranePlanError(rc, load().cp_last_error().decode())


def _ptr(t) -> Optional[int]:
    """Device pointer of a CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _c4(v) -> ctypes.Array:
    a = np.ascontiguousarray(v, dtype=np.float64).reshape(4)
    return (ctypes.c_double * 4)(*a.tolist())


# --------------------------------------------------------------------------- marshalling

def make_model(crane) -> cp_model:
    """cp_model from a workloads.CraneModel."""
    m = cp_model()
    m.base_z, m.boom_len, m.jib_len = crane.base_z, crane.boom_len, crane.jib_len
    for j in range(4):
        m.q_min[j], m.q_max[j] = crane.q_min[j], crane.q_max[j]
    if len(crane.spheres) > CP_MAX_SPHERES:
        raise ValueError("at most %d spheres" % CP_MAX_SPHERES)
    m.n_spheres = len(crane.spheres)
    for s, sp in enumerate(crane.spheres):
        m.spheres[s] = cp_sphere(sp.link, sp.offset, sp.radius)
    return m


class HostScene:
    """cp_scene over host arrays (keeps them alive)."""

    def __init__(self, cylinders, boxes):
        cyl = np.ascontiguousarray(cylinders, dtype=np.float64).reshape(-1, 5)
        box = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 6)
        self.cyl, self.box = cyl, box
        self.c = cp_scene(cyl.shape[0], cyl.ctypes.data if cyl.shape[0] else None,
                          box.shape[0], box.ctypes.data if box.shape[0] else None)

    @classmethod
    def from_scene(cls, scene) -> "HostScene":
        return cls(scene.cylinders, scene.boxes)


def make_params(N: int, K: int, S: int, n_elites: int = 0, w_c: float = 100.0,
                w_l: float = 100.0, lambda_c: float = 1.0, sigma: float = 1.0,
                eps: float = 1e-8, init_std_frac: float = 0.1, seed: int = 0, query: int = 0,
                max_cylinders: int = 0, max_boxes: int = 0, grid_cell: float = 0.0,
                grid_half_extent: float = 0.0, max_grid_items: int = 0,
                smooth_margin: float = 0.05, smooth_beta: float = 0.01,
                eval_ctas_per_sm: int = 0, debug_withhold_staging: int = 0,
                eval_exhaustive: int = 0, update_rule: int = CP_UPDATE_PAPER,
                sampler: int = CP_SAMPLE_FACTOR, collision_model: int = CP_COLLISION_SPHERES) -> cp_params:
    return cp_params(N, K, S, n_elites, w_c, w_l, lambda_c, sigma, eps, init_std_frac, seed,
                     query, max_cylinders, max_boxes, grid_cell, grid_half_extent,
                     max_grid_items, smooth_margin, smooth_beta, eval_ctas_per_sm,
                     debug_withhold_staging, eval_exhaustive, update_rule, collision_model, sampler)


# --------------------------------------------------------------------------- entry points

def cp_last_error() -> str:
    return load().cp_last_error().decode()


def cp_version() -> int:
    return int(load().cp_version())


def cp_launch_count() -> int:
    return int(load().cp_launch_count())


def cp_debug_fail_allocations(n: int) -> None:
    load().cp_debug_fail_allocations(int(n))


def cp_debug_static_withhold_staging(on: bool) -> None:
    load().cp_debug_static_withhold_staging(1 if on else 0)


def cp_plan_init(model: cp_model, scene: HostScene, params: cp_params, stream=None) -> int:
    """Returns the planner handle (an opaque pointer as int)."""
    out = _P()
    _check(load().cp_plan_init(ctypes.byref(model), ctypes.byref(scene.c), ctypes.byref(params),
                               _stream(stream), ctypes.byref(out)))
    return out.value


def cp_destroy(p: int) -> None:
    load().cp_destroy(p)


def cp_set_scene(p: int, scene: HostScene) -> None:
    _check(load().cp_set_scene(p, ctypes.byref(scene.c)))


def cp_set_endpoints(p: int, q0, qd) -> None:
    _check(load().cp_set_endpoints(p, _c4(q0), _c4(qd)))


def cp_sample(p: int, it: int, xi) -> None:
    _check(load().cp_sample(p, int(it), _ptr(xi)))


def cp_evaluate(p: int, xi, n: int, J, flag=None, terms=None, substep_flags=None,
                pen=None) -> None:
    _check(load().cp_evaluate(p, _ptr(xi), int(n), _ptr(J), _ptr(flag), _ptr(terms),
                              _ptr(substep_flags), _ptr(pen)))


def cp_update(p: int, J, xi) -> None:
    _check(load().cp_update(p, _ptr(J), _ptr(xi)))


def cp_synchronize(p: int) -> None:
    _check(load().cp_synchronize(p))


def cp_plan(p: int, iters: int, K: Optional[int] = None):
    """Returns (control points double[K+8][4] or None, stats dict)."""
    stats = cp_plan_stats()
    ctrl = np.zeros((K + 8, 4)) if K is not None else None
    cptr = ctrl.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if ctrl is not None else None
    _check(load().cp_plan(p, int(iters), cptr, ctypes.byref(stats)))
    return ctrl, {f: getattr(stats, f) for f, _ in cp_plan_stats._fields_}


def cp_signed_distance(p: int, q, n: int, d) -> None:
    _check(load().cp_signed_distance(p, _ptr(q), int(n), _ptr(d)))


def cp_forward_kinematics(p: int, q, n: int, centres=None, tip=None) -> None:
    _check(load().cp_forward_kinematics(p, _ptr(q), int(n), _ptr(centres), _ptr(tip)))


def make_hull_model(w=(0.2, 0.2, 0.15), h=(0.2, 0.2, 0.15), pad: float = 0.2, grapple_w: float = 0.25,
                    grapple_len: float = 1.0) -> cp_hull_model:
    return cp_hull_model((ctypes.c_double * 3)(*w), (ctypes.c_double * 3)(*h), pad, grapple_w, grapple_len)


def cp_hull_penetration(p: int, q, n: int, pen, hulls: Optional[cp_hull_model] = None) -> None:
    _check(load().cp_hull_penetration(p, _ptr(q), int(n), ctypes.byref(hulls) if hulls is not None else None,
                                      _ptr(pen)))


def cp_set_hull_model(p: int, hulls: Optional[cp_hull_model] = None) -> None:
    _check(load().cp_set_hull_model(p, ctypes.byref(hulls) if hulls is not None else None))


def make_ik_params(lambda_q: float = 1.0, lambda_c: float = 1.0, grapple_len: float = 1.0,
                   mu0: float = 1e-3, seed: int = 0, query: int = 0, restarts: int = 8,
                   iters: int = 50) -> cp_ik_params:
    return cp_ik_params(lambda_q, lambda_c, grapple_len, mu0, seed, query, restarts, iters)


def cp_ik(p: int, targets, n: int, ik: cp_ik_params, q, f, q_init=None, restart=None,
          r=None) -> None:
    _check(load().cp_ik(p, _ptr(targets), int(n), ctypes.byref(ik), _ptr(q_init), _ptr(q),
                        _ptr(f), _ptr(restart), _ptr(r)))


def cp_get_distribution(p: int, mu=None, C=None) -> None:
    _check(load().cp_get_distribution(p, _ptr(mu), _ptr(C)))


def cp_set_distribution(p: int, mu, C, it: int) -> None:
    _check(load().cp_set_distribution(p, _ptr(mu), _ptr(C), int(it)))


def cp_get_factor(p: int, L) -> None:
    _check(load().cp_get_factor(p, _ptr(L)))


def cp_get_cma_state(p: int, state) -> None:
    _check(load().cp_get_cma_state(p, _ptr(state)))


def cp_set_cma_state(p: int, state) -> None:
    _check(load().cp_set_cma_state(p, _ptr(state)))


def cp_get_elites(p: int, idx) -> None:
    _check(load().cp_get_elites(p, _ptr(idx)))


def cp_set_metrics(p: int, on: bool) -> None:
    _check(load().cp_set_metrics(p, 1 if on else 0))


def cp_get_metrics(p: int, max_rows: int = 256) -> np.ndarray:
    """Rows {iteration, best J, mean J, tr C, collision-free fraction}, oldest first."""
    buf = np.zeros((max(max_rows, 1), 5), dtype=np.float64)
    n = ctypes.c_int32()
    _check(load().cp_get_metrics(p, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(max_rows),
                                 ctypes.byref(n)))
    return buf[: n.value].copy()


def cp_get_population(p: int, xi=None, J=None) -> None:
    _check(load().cp_get_population(p, _ptr(xi) if xi is not None else None,
                                    _ptr(J) if J is not None else None))


def cp_philox4x32_10(ctr, key: int, n: int, out, stream=None) -> None:
    _check(load().cp_philox4x32_10(_ptr(ctr), int(key), int(n), _ptr(out), _stream(stream)))


def cp_evaluate_static(model: cp_model, cyl, n_cyl: int, box, n_box: int, K: int, S: int,
                       w_c: float, w_l: float, lambda_c: float, q0, qd, xi, n: int, J,
                       flag=None, terms=None, stream=None) -> None:
    """Evaluation without device allocation (fixed library scratch). cyl is a CUDA float64
    tensor [n_cyl][5] (cx, cy, R, z_lo, z_hi), box a CUDA float64 tensor [n_box][6]."""
    _check(load().cp_evaluate_static(ctypes.byref(model), _ptr(cyl), int(n_cyl), _ptr(box),
                                     int(n_box), int(K), int(S), float(w_c), float(w_l),
                                     float(lambda_c), _c4(q0), _c4(qd), _ptr(xi), int(n),
                                     _ptr(J), _ptr(flag), _ptr(terms), _stream(stream)))


def cp_smooth_cost(p: int, xi, n: int, J) -> None:
    _check(load().cp_smooth_cost(p, _ptr(xi), int(n), _ptr(J)))


def cp_smooth_cost_grad(p: int, xi, n: int, gJ, J, dxi) -> None:
    _check(load().cp_smooth_cost_grad(p, _ptr(xi), int(n), _ptr(gJ), _ptr(J), _ptr(dxi)))


def cp_polish(p: int, xi, n: int, steps: int, alpha: float) -> None:
    _check(load().cp_polish(p, _ptr(xi), int(n), int(steps), float(alpha)))


def cp_batch_init(model: cp_model, scenes, params, q0s, qds, iters: int) -> int:
    """scenes: HostScene per query; params: cp_params per query; returns the batch handle."""
    nq = len(scenes)
    qs = (cp_query * nq)()
    for i in range(nq):
        qs[i].scene = scenes[i].c
        qs[i].params = params[i]
        qs[i].q0 = _c4(q0s[i])
        qs[i].qd = _c4(qds[i])
    out = _P()
    _check(load().cp_batch_init(ctypes.byref(model), qs, nq, int(iters), ctypes.byref(out)))
    return out.value


def cp_batch_set_endpoints(b: int, q: int, q0, qd) -> None:
    _check(load().cp_batch_set_endpoints(b, int(q), _c4(q0), _c4(qd)))


def cp_batch_run(b: int, nq: int, K=None):
    """Runs the batch; returns [(ctrl [K+8][4] or None, stats dict)] per query."""
    res = (cp_batch_result * nq)()
    _check(load().cp_batch_run(b, res))
    out = []
    for i in range(nq):
        st = {f: getattr(res[i].stats, f) for f, _ in cp_plan_stats._fields_}
        ctrl = None
        if K is not None:
            k = K[i]
            ctrl = np.ctypeslib.as_array(res[i].ctrl)[: 4 * (k + 8)].reshape(k + 8, 4).copy()
        out.append((ctrl, st))
    return out


def cp_batch_planner(b: int, q: int) -> int:
    return load().cp_batch_planner(b, int(q))


def cp_batch_set_shape(b: int, threads: int = 256, ctas_per_sm: int = 0, items_per_warp: int = 2) -> None:
    sh = cp_batch_shape(int(threads), int(ctas_per_sm), int(items_per_warp))
    _check(load().cp_batch_set_shape(b, ctypes.byref(sh)))


def cp_batch_evaluate(b: int, reps: int = 3) -> float:
    """Mean duration (ms) of the batched evaluation launch over the current populations."""
    ms = ctypes.c_double()
    _check(load().cp_batch_evaluate(b, int(reps), ctypes.byref(ms)))
    return ms.value


def cp_batch_get_info(b: int) -> dict:
    info = cp_batch_info()
    _check(load().cp_batch_get_info(b, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in cp_batch_info._fields_}


def cp_batch_destroy(b: int) -> None:
    load().cp_batch_destroy(b)


def cp_set_timing(p: int, on: bool) -> None:
    _check(load().cp_set_timing(p, 1 if on else 0))


def cp_get_timing(p: int) -> dict:
    t = cp_timing()
    _check(load().cp_get_timing(p, ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in cp_timing._fields_}


def cp_traj_init(model: cp_model, tp: cp_traj_params, max_paths: int, stream=None) -> int:
    """Returns the trajectory solver handle (an opaque pointer as int)."""
    out = _P()
    _check(load().cp_traj_init(ctypes.byref(model), ctypes.byref(tp), int(max_paths), _stream(stream),
                               ctypes.byref(out)))
    return out.value


def cp_traj_destroy(t: int) -> None:
    load().cp_traj_destroy(t)


def cp_traj_targets(t: int, ctrl, K: int, n: int, q_star) -> None:
    _check(load().cp_traj_targets(t, _ptr(ctrl), int(K), int(n), _ptr(q_star)))


def cp_traj_initial_guess(t: int, q_star, n: int, z) -> None:
    _check(load().cp_traj_initial_guess(t, _ptr(q_star), int(n), _ptr(z)))


def cp_traj_step(t: int, q_star, n: int, z, lam, mu: float, dz) -> None:
    _check(load().cp_traj_step(t, _ptr(q_star), int(n), _ptr(z), _ptr(lam), float(mu), _ptr(dz)))


def cp_traj_solve(t: int, q_star, n: int, z, stats) -> None:
    _check(load().cp_traj_solve(t, _ptr(q_star), int(n), _ptr(z), _ptr(stats)))


def cp_alu_peaks() -> dict:
    """Measured FP32 and FP64 FMA throughput of the current device, TFLOP/s."""
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    _check(load().cp_alu_peaks(ctypes.byref(f32), ctypes.byref(f64)))
    return {"fp32_tflops": f32.value, "fp64_tflops": f64.value}


class Planner:
    """Owns one planner handle and the host scene it was created from."""

    def __init__(self, crane, scene, params: cp_params, stream=None):
        self.model = make_model(crane)
        self.scene = HostScene.from_scene(scene)
        self.params = params
        self.N, self.K, self.S = params.n_candidates, params.n_waypoints, params.substeps
        self.D = 4 * self.K
        self.n_s = (self.K + 3) * self.S
        self.nu = params.n_elites if params.n_elites > 0 else self.N // 2
        self.handle = cp_plan_init(self.model, self.scene, params, stream)

    def close(self):
        if self.handle:
            cp_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

"""Benchmark of the stochastic B-spline path optimisation on one GB300 per rank.

A step is one whole plan: the T iterations of Algorithm 1 (sample, evaluate, rank,
update; arXiv 2503.14160 Sec. 4.1) for one query, then the evaluation of the mean path.
Default workload: the dense forest (N = 65536 candidates, K = 32 waypoints, S = 128
checkpoints per span, 5000 trees at >= 0.8 m spacing in a 2-50 m annulus plus 50 boxes,
through a polar obstacle index with 0.5 m rings, 200 iterations), synthetic and seeded; --workload
single_large runs the single large query (N = 4096, K = 16, S = 64, 500 trees, 100
iterations).

Metric: candidate paths evaluated per second = N * T / (time per plan), plus ms per plan.
  value  device time of the plan on the planner's stream (CUDA events), inputs resident
  e2e    wall time through the C ABI with host buffers: scene and end points copied in,
         control points and statistics copied out, every step

--impl reference times the FP64 CPU oracle (the checker) on the host cores on a bounded
sample of the same workload. Under torchrun every rank runs an independent replica
(its own query, Philox query word = rank); value sums the ranks' candidates over the
slowest rank's time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate paths evaluated/sec & ms per plan on 1 GB300 vs FP64 CPU oracle"
UNIT = "candidate paths/s"
WORKLOAD = "dense_forest"
PEAK_SM_COUNT = 152
FP32_LANES_PER_SM = 128
FLOPS_PER_PAIR = 5          # 2 sub, 1 mul, 1 fma per sphere-obstacle pair
FLOPS_PER_CHECKPOINT = 140  # spline 32, kinematics ~80, length 12, limits 16
FLOPS_FRAME_PER_SPHERE = 6  # broad phase: the sphere centre in the unit's frame (2 mul, 2 fma)
FLOPS_PER_BROAD_TEST = 10   # broad phase: one obstacle against a unit's box
FLOPS_PER_INDEX_TEST = 8    # polar index: a listed obstacle in a lane's plane (p, q, bound)
FLOPS_PER_PACKED_PAIR = 3   # polar index: one sphere's filter in the packed test (FP32x2 add + fma)
FP32_PEAK_TFLOPS = PEAK_SM_COUNT * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12


def eval_roofline(timing, n_spheres, n_obstacles, n_s, candidates, form, sm_mhz):
    """Algorithmic FP32 work of the evaluation launches in `timing` over their device time.

    Per checkpoint FLOPS_PER_CHECKPOINT (spline, kinematics, length, limits); per sphere and
    obstacle whose pair test runs FLOPS_PER_PAIR. form "exhaustive": every obstacle of every
    unit is tested. "broad": every (unit, obstacle) takes one box test, each checkpoint
    places its spheres in the unit frame, and only the counted survivors take pair tests.
    "polar": every obstacle listed for a checkpoint's slew angle and reach (counted on the
    device) is placed in the checkpoint's plane and takes the filter for each sphere; pair
    tests are those sphere filters."""
    units = timing["eval_units"]
    pairs = timing["eval_pair_tests"]
    if units <= 0 or pairs < 0 or timing["eval_ms"] <= 0:
        return None
    flops = candidates * n_s * FLOPS_PER_CHECKPOINT
    flops += pairs * (FLOPS_PER_PACKED_PAIR if form == "polar" else FLOPS_PER_PAIR)
    if form == "broad":
        flops += candidates * n_s * n_spheres * FLOPS_FRAME_PER_SPHERE
        flops += units * n_obstacles * FLOPS_PER_BROAD_TEST
    elif form == "polar":
        flops += max(timing.get("eval_box_tests", 0), 0) * FLOPS_PER_INDEX_TEST
    achieved = flops / (timing["eval_ms"] / 1e3) / 1e12
    kernel = {"broad": "k_eval_broad", "exhaustive": "k_eval", "polar": "k_eval_polar"}[form]
    return {"bound": "alu", "kernel": kernel,
            "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS,
            "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
            "frac_at_observed_clock": (achieved / (FP32_PEAK_TFLOPS * sm_mhz / 2070.0)
                                       if sm_mhz else None),
            "eval_ms_per_launch": timing["eval_ms"] / max(timing["eval_launches"], 1),
            "eval_launches": timing["eval_launches"],
            "pair_tests_per_checkpoint": pairs / max(candidates * n_s, 1),
            "listed_obstacles_per_checkpoint": (timing["eval_box_tests"] / max(candidates * n_s, 1)
                                                if timing.get("eval_box_tests", -1) >= 0 else None),
            "pair_tests_exhaustive_per_checkpoint": n_spheres * n_obstacles}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def steps_for_clocks(steps, run_once, min_seconds=1.0):
    """Timed steps for a workload whose step takes well under a clock sample period: at
    least `steps`, and enough that the timed region lasts min_seconds, so that the clock
    sampler (one reading every 200 ms) sees it under load. Untimed steps measure it."""
    import torch
    dt = float("inf")
    for _ in range(3):   # the shortest of three: the first call can carry one-off costs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_once()
        torch.cuda.synchronize()
        dt = min(dt, time.perf_counter() - t0)
    return max(steps, int(math.ceil(min_seconds / max(dt, 1e-6))))


KERNEL_SOURCES = {
    "k_eval_broad": ("k_eval.cu", "eval_common.cuh", "cp_internal.cuh"),
    "k_eval_polar": ("k_grid.cu", "eval_common.cuh", "cp_internal.cuh"),
}

# DRAM bytes (read + write) per launch of an evaluation kernel from one ncu capture of the
# workload's launch (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the SHA-1 of the
# kernel's sources at the time of the capture: reported only while the sources still hash
# to it, None once the kernel has changed.
PROFILED_TRAFFIC = {
    # captured at b833554f...; the file changed since only in the batched kernel's call of the
    # item body, which leaves k_eval_polar as it was
    ("k_eval_polar", "dense_forest"): {"sha1": "8484a179acebfd8666a344e6c3f694ae59bae607", "bytes": 34001408.0},
    ("k_eval_polar", "single_large"): {"sha1": "8484a179acebfd8666a344e6c3f694ae59bae607", "bytes": 1160192.0},
}


def kernel_source_sha1(kernel):
    """SHA-1 over the sources of an evaluation kernel: its .cu file and eval_common.cuh whole,
    and cp_internal.cuh up to its first launcher declaration (the device records the kernel
    reads; the host-side declarations after it do not change the kernel)."""
    import hashlib
    h = hashlib.sha1()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2503_14160_gb300", "csrc", name), "rb") as f:
            data = f.read()
        if name == "cp_internal.cuh":
            data = data[:data.index(b"int launch_eval(")]
        h.update(data)
    return h.hexdigest()


def traffic_per_launch(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from its last ncu capture, or None
    when there is none for this workload or the kernel's sources have changed since."""
    rec = PROFILED_TRAFFIC.get((kernel, workload))
    if rec is None or rec["sha1"] != kernel_source_sha1(kernel):
        return None
    return rec["bytes"]


def select_endpoints_gpu(cp, planner, crane, seed, query):
    """Start/goal by the rule of the workload, using the library's d(q) kernel."""
    import torch
    from paper_2503_14160_gb300 import workloads

    def dist(q):
        qt = torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
        d = torch.zeros(q.shape[0], dtype=torch.float32, device="cuda")
        cp.cp_signed_distance(planner.handle, qt, q.shape[0], d)
        return d.cpu().numpy().astype(np.float64)

    q0, qd, ok, _ = workloads.select_endpoints(crane, dist, seed=seed, query=query)
    return q0, qd, ok


def max_over_ranks(values, device):
    """Each value's maximum over the ranks of the process group (the slowest replica);
    the values themselves on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(units_per_rank, world_size, ms_slowest):
    """Whole-job throughput of independent replicas: every rank's units over the slowest
    rank's time."""
    return units_per_rank * world_size / (ms_slowest / 1e3)


def flush_l2(buf):
    buf.add_(1.0)   # a write of a buffer larger than the 129 MB L2


def resolve_sampler(args, wl):
    """Step (1): the FP64 Cholesky factor, or the factor-free draw from the last update's
    elites (the same distribution; paper rule only). "auto" takes the elites where their
    N x nu x D FP32 product is cheaper than the FP64 moments and factor it replaces."""
    if args.sampler != "auto":
        return args.sampler
    if args.update_rule != "paper":
        return "factor"
    N, D = wl.n_candidates, 4 * wl.n_waypoints
    return "elites" if N * (N // 2) * D <= 2 ** 31 else "factor"


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2503_14160_gb300 import build, craneplan as cp, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    # a stream of our own: cp_plan records its iterations as a CUDA graph there (the legacy
    # default stream cannot be captured); every event below sits on this stream
    torch.cuda.set_stream(torch.cuda.Stream())
    build.build()
    cp.load()
    wl = workloads.WORKLOADS[args.workload]
    iters = args.iterations or wl.iterations
    crane = workloads.forestry_crane()
    scene = workloads.make_scene(wl)
    sampler = resolve_sampler(args, wl)
    grid_cell = 0.0 if args.exhaustive else wl.grid_cell   # the exhaustive form takes no index
    params = cp.make_params(wl.n_candidates, wl.n_waypoints, wl.substeps, seed=wl.seed, query=rank,
                            grid_cell=grid_cell, eval_exhaustive=int(args.exhaustive),
                            update_rule=cp.CP_UPDATE_CMAES if args.update_rule == "cmaes" else cp.CP_UPDATE_PAPER,
                            sampler=cp.CP_SAMPLE_ELITES if sampler == "elites" else cp.CP_SAMPLE_FACTOR,
                            collision_model=cp.CP_COLLISION_HULLS if args.collision == "hulls" else cp.CP_COLLISION_SPHERES)
    planner = cp.Planner(crane, scene, params)
    h = planner.handle
    q0, qd, ok = select_endpoints_gpu(cp, planner, crane, wl.seed, rank)
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB

    def barrier():
        if ws > 1:
            dist.barrier()

    # warm-up plans
    for _ in range(args.warmup):
        cp.cp_set_endpoints(h, q0, qd)
        cp.cp_plan(h, iters, K=wl.n_waypoints)
    torch.cuda.synchronize()

    # device-timed plans (inputs resident): events around each plan, L2 flushed between
    times = []
    launches0 = cp.cp_launch_count()
    stats = None
    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush_l2(flush)
            start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            start.record(stream)
            cp.cp_set_endpoints(h, q0, qd)
            _, stats = cp.cp_plan(h, iters, K=None)
            end.record(stream)
            end.synchronize()
            times.append(start.elapsed_time(end))
        torch.cuda.synchronize()
        barrier()
    launches = cp.cp_launch_count() - launches0

    # the same plans again with per-stage events and the work counters on (outside the
    # timed region: the stage events add a little device time of their own)
    # (at most 3 and 5 plans: the dense forest's plans take seconds each)
    cp.cp_set_timing(h, True)
    n_timing = min(args.steps, 3)
    for _ in range(n_timing):
        flush_l2(flush)
        cp.cp_set_endpoints(h, q0, qd)
        cp.cp_plan(h, iters, K=None)
    timing = cp.cp_get_timing(h)
    cp.cp_set_timing(h, False)
    # one more plan with the per-iteration metrics on (outside the timed region)
    cp.cp_set_metrics(h, True)
    cp.cp_set_endpoints(h, q0, qd)
    cp.cp_plan(h, iters, K=None)
    metric_rows = cp.cp_get_metrics(h)
    cp.cp_set_metrics(h, False)
    picks = sorted({0, len(metric_rows) // 4, len(metric_rows) // 2, 3 * len(metric_rows) // 4, len(metric_rows) - 1})
    iteration_metrics = {"columns": ["iteration", "best_J", "mean_J", "trace_C", "collision_free_fraction"],
                         "rows": [[float(v) for v in metric_rows[i]] for i in picks if 0 <= i < len(metric_rows)]}

    # end-to-end through the C ABI with host buffers, wall clock
    e2e_times = []
    for _ in range(min(args.steps, 5)):
        flush_l2(flush)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        cp.cp_set_scene(h, planner.scene)
        cp.cp_set_endpoints(h, q0, qd)
        ctrl, st = cp.cp_plan(h, iters, K=wl.n_waypoints)
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    barrier()

    ms, ms_e2e = max_over_ranks([float(np.mean(times)), float(np.mean(e2e_times))], "cuda")
    units = wl.n_candidates * iters * ws
    value = job_throughput(wl.n_candidates * iters, ws, ms)

    # roofline of the evaluation kernel (FK + collision + cost); per plan the kernel runs
    # T times on N candidates and once on the mean path
    n_s = wl.n_checkpoints
    eval_ms = timing["eval_ms"] / max(timing["eval_launches"], 1)
    clk = clocks.summary()
    candidates = n_timing * (wl.n_candidates * iters + 1)
    roofline_exhaustive = None
    peaks_fp64 = None
    form = "polar" if grid_cell > 0 else ("exhaustive" if args.exhaustive else "broad")
    if args.collision == "hulls":
        # the hull form's work per checkpoint depends on the pairs its scan keeps; its line
        # reports the launch time only
        roofline = {"bound": "alu", "kernel": "k_eval_hulls", "achieved": None, "peak": None, "unit": "TFLOP/s",
                    "frac": None, "traffic": None,
                    "eval_ms_per_launch": timing["eval_ms"] / max(timing["eval_launches"], 1)}
    else:
        roofline = eval_roofline(timing, len(crane.spheres), scene.n_cyl + scene.n_box, n_s,
                                 candidates, form, clk.get("sm_mhz"))
    if roofline is not None and roofline.get("achieved") is not None:
        roofline["traffic"] = traffic_per_launch(roofline["kernel"], wl.name)
        roofline["traffic_source"] = (
            "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (iteration 0) of this "
            "kernel's current source on this workload, taken in a separate profiling run"
            if roofline["traffic"] is not None else
            "none: no ncu capture of this kernel's current source on this workload")
        peaks = cp.cp_alu_peaks()
        peaks_fp64 = peaks["fp64_tflops"]
        roofline["measured_fma_peaks"] = peaks
        roofline["frac_of_measured_fp32"] = roofline["achieved"] / peaks["fp32_tflops"]
    if args.collision == "spheres" and scene.n_cyl + scene.n_box <= 1000:
        if not args.exhaustive:
            roofline_exhaustive = exhaustive_roofline(cp, crane, scene, wl, q0, qd,
                                                      clk.get("sm_mhz"))

    if rank == 0:
        bi = scene.n_cyl * 40 + scene.n_box * 48 + 64
        bo = (wl.n_waypoints + 8) * 32 + 6 * 8 + 4
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded crane-and-forest scene; paper environments unavailable)",
            "config": {"workload": "%s: N=%d K=%d S=%d cylinders=%d iterations=%d per plan"
                                   % (wl.name, wl.n_candidates, wl.n_waypoints, wl.substeps,
                                      scene.n_cyl, iters),
                       "step": "one plan", "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "flushed between steps (256 MB write)",
                       "endpoints_ok": bool(ok), "update_rule": args.update_rule, "sampler": sampler,
                       "collision_model": args.collision},
            "ms_per_plan": ms,
            "e2e": {"value": units / (ms_e2e / 1e3), "unit": UNIT, "ms_per_plan": ms_e2e,
                    "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
            "gpu_launches": launches,
            "roofline": roofline,
            "roofline_exhaustive": roofline_exhaustive,
            "eval_kernel": {"name": "k_eval_hulls" if args.collision == "hulls" else
                            {"broad": "k_eval_broad", "exhaustive": "k_eval", "polar": "k_eval_polar"}[form],
                            "ms_per_launch": eval_ms, "launches": timing["eval_launches"]},
            "stage_ms_per_plan": {k.replace("_ms", ""): timing[k] / n_timing
                                  for k in ("eval_ms", "sample_ms", "factor_ms", "update_ms")},
            "fp64_stages": fp64_stages(timing, wl, peaks_fp64, sampler),
            "sampler_stage": sampler_stage(timing, wl, sampler),
            "plan_result": {"J": stats["J"], "length": stats["length"], "flag": stats["flag"]},
            "iteration_metrics": iteration_metrics,
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            # the CPU-baseline leg: the oracle timed on the host cores, and the error of the
            # results above against it
            ctrl_last, st_last = cp.cp_plan(h, 0, K=wl.n_waypoints)   # the plan's mean path, again
            line["oracle_error"] = oracle_errors(cp, h, wl, crane, scene, q0, qd, ctrl_last, st_last, iters)
            line["cpu_baseline"] = cpu_baseline(wl, crane, scene, q0, qd, args.cpu_seconds,
                                                single_core_seconds=args.cpu_seconds / 4)
        print(json.dumps(line), flush=True)
    planner.close()
    if ws > 1:
        dist.destroy_process_group()


def fp64_stages(timing, wl, fp64_peak, sampler):
    """The FP64 stages against the measured FP64 FMA rate: the Cholesky factor (D^3/3 FMAs per
    call) and the update (nu D(D+1)/2 FMAs for the covariance plus nu D for the mean; with
    the factor-free sampler only the mean is FP64), FMA = 2 flops."""
    if not fp64_peak or timing["factor_launches"] <= 0 or timing["update_launches"] <= 0:
        return None
    D = 4 * wl.n_waypoints
    nu = wl.n_candidates // 2
    f_factor = 2.0 * D ** 3 / 3.0
    f_update = 2.0 * (nu * D if sampler == "elites" else nu * D * (D + 1) / 2.0 + nu * D)
    ms_f = timing["factor_ms"] / timing["factor_launches"]
    ms_u = timing["update_ms"] / timing["update_launches"]
    out = {}
    for name, fl, ms in (("factor", f_factor, ms_f), ("update", f_update, ms_u)):
        achieved = fl / (ms / 1e3) / 1e12
        out[name] = {"bound": "fp64", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak, "peak_basis": "cp_alu_peaks (measured FP64 FMA rate)",
                     "us_per_call": ms * 1e3}
    return out


def sampler_stage(timing, wl, sampler):
    """The sampling stage with the factor-free sampler: the product of N x nu normals and the
    nu x D' scaled elite deviations (D' = D rounded up to 16) on the tensor cores as three
    TF32 products (3 x 2 N nu D' flops), against the TF32 rate taken as the measured BF16
    GEMM rate x 1.1 / 2.25 (the nominal dense TF32 : BF16 ratio). The stage is bound by
    generating the N (nu + D) normals (Philox and Box-Muller on the FP32 and integer pipes),
    so its tensor fraction is low by construction."""
    if sampler != "elites" or timing["sample_launches"] <= 0:
        return None
    D = 4 * wl.n_waypoints
    Dp = (D + 15) // 16 * 16
    nu = wl.n_candidates // 2
    us = timing["sample_ms"] / timing["sample_launches"] * 1e3
    flops = 3 * 2.0 * wl.n_candidates * nu * Dp
    bf16 = measured_peaks().get("bf16_tflops_sustained")
    basis = "sustained BF16 GEMM of measured peaks x 1.1/2.25 (nominal TF32:BF16)"
    if not bf16:
        # no measured peaks on this machine: the earlier GB300 measurement of a sustained
        # BF16 GEMM (about 1.7 PFLOP/s under the power cap) stands in, labelled as such
        bf16 = 1700.0
        basis = "fallback sustained BF16 GEMM of 1700 TFLOP/s x 1.1/2.25 (nominal TF32:BF16)"
    out = {"kernels": "k_sample_elites (tcgen05 kind::tf32, 3xTF32 split) + k_sample_reduce",
           "us_per_call": us,
           "normals_per_s": wl.n_candidates * (nu + D) / (us / 1e6)}
    achieved = flops / (us / 1e6) / 1e12
    peak = bf16 * 1.1 / 2.25
    out["tensor"] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "peak_basis": basis}
    return out


def exhaustive_roofline(cp, crane, scene, wl, q0, qd, sm_mhz, iterations=10):
    """The exhaustive form of the evaluation (every sphere against every obstacle) timed on
    the same query for a few iterations, for comparison with the culled forms."""
    import torch
    params = cp.make_params(wl.n_candidates, wl.n_waypoints, wl.substeps, seed=wl.seed,
                            eval_exhaustive=1)
    planner = cp.Planner(crane, scene, params)
    try:
        h = planner.handle
        cp.cp_set_endpoints(h, q0, qd)
        cp.cp_plan(h, 2, K=None)
        torch.cuda.synchronize()
        cp.cp_set_timing(h, True)
        cp.cp_set_endpoints(h, q0, qd)
        cp.cp_plan(h, iterations, K=None)
        t = cp.cp_get_timing(h)
        cp.cp_set_timing(h, False)
    finally:
        planner.close()
    r = eval_roofline(t, len(crane.spheres), scene.n_cyl + scene.n_box, wl.n_checkpoints,
                      wl.n_candidates * iterations + 1, "exhaustive", sm_mhz)
    if r is not None:
        r["iterations"] = iterations
    return r


def run_differentiable(args):
    """The differentiable form: adjoint of the smooth cost for N candidates (gradients/s),
    and 10 gradient-descent polish steps on the 64 best candidates of a sampled population."""
    import torch
    from paper_2503_14160_gb300 import build, craneplan as cp, workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    cp.load()
    wl = workloads.WORKLOADS["differentiable"]
    crane = workloads.forestry_crane()
    scene = workloads.make_scene(wl)
    params = cp.make_params(wl.n_candidates, wl.n_waypoints, wl.substeps, seed=wl.seed)
    planner = cp.Planner(crane, scene, params)
    h = planner.handle
    q0, qd, ok = select_endpoints_gpu(cp, planner, crane, wl.seed, rank)
    cp.cp_set_endpoints(h, q0, qd)
    N, K = wl.n_candidates, wl.n_waypoints
    xi = torch.zeros(N, K, 4, device="cuda")
    J = torch.zeros(N, dtype=torch.float64, device="cuda")
    dxi = torch.zeros_like(xi)
    cp.cp_sample(h, 0, xi)
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        cp.cp_smooth_cost_grad(h, xi, N, None, J, dxi)
    steps = steps_for_clocks(args.steps, lambda: (flush_l2(flush), cp.cp_smooth_cost_grad(h, xi, N, None, J, dxi)))
    times = []
    l0 = cp.cp_launch_count()
    with ClockSampler(local) as clocks:
        for _ in range(steps):
            flush_l2(flush)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            cp.cp_smooth_cost_grad(h, xi, N, None, J, dxi)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
    launches = cp.cp_launch_count() - l0
    ms = float(np.mean(times))
    # polish: 64 best of the population, 10 steps, alpha = 1e-3
    cp.cp_evaluate(h, xi, N, J)
    best = xi[torch.argsort(J)[:64]].contiguous()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    cp.cp_polish(h, best, 64, 10, 1e-3)
    b.record(stream)
    b.synchronize()
    polish_ms = a.elapsed_time(b)
    # end to end: candidates copied in from pinned host memory, gradients copied out
    host_xi = xi.cpu().pin_memory()
    host_g = torch.empty_like(host_xi).pin_memory()
    e2e = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xi.copy_(host_xi, non_blocking=True)
        cp.cp_smooth_cost_grad(h, xi, N, None, J, dxi)
        host_g.copy_(dxi, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    line = {"metric": "candidate gradients/sec (adjoint of the smooth path cost)",
            "value": N / (ms / 1e3), "unit": "gradients/s", "n_gpus": ws, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded crane-and-forest scene)",
            "config": {"workload": "differentiable: N=%d K=%d S=%d cylinders=%d, softplus margin "
                                   "0.05 m" % (N, K, wl.substeps, scene.n_cyl),
                       "step": "one adjoint launch over all candidates",
                       "l2": "flushed between steps (256 MB write)"},
            "polish_ms": polish_ms, "polish": "64 best candidates x 10 steps, alpha 1e-3",
            "e2e": {"value": N / (float(np.mean(e2e)) / 1e3), "unit": "gradients/s",
                    "h2d_bytes_per_step": N * K * 16, "d2h_bytes_per_step": N * K * 16},
            "gpu_launches": launches, "clocks": clocks.summary()}
    if not args.no_cpu_baseline:
        sys.path.insert(0, os.path.join(ROOT, "oracle"))
        import oracle
        oracle.set_threads(os.cpu_count() or 1)
        pb = oracle.Problem(crane, scene, oracle.CostParams(K=K, S=wl.substeps))
        x = xi[:2 * (os.cpu_count() or 1)].cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        oracle.smooth_grad(pb, x, q0, qd)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": x.shape[0] / el, "unit": "gradients/s",
                                "cores": oracle.get_threads(), "kind": "oracle",
                                "sample": "%d analytic FP64 gradients" % x.shape[0]}
    print(json.dumps(line), flush=True)
    planner.close()


IK_TARGETS, IK_RESTARTS, IK_ITERS = 16384, 8, 50
IK_FLOPS_PER_EVAL = 150     # kinematics of 12 spheres and the tip, the residual
IK_FLOPS_PER_OBSTACLE = 4   # plane test of one obstacle (part of its 2 fma + 3 mul)
IK_FLOPS_PER_SOLVE = 200    # Jacobian rows, J^T J, J^T r, damping, 4x4 Cholesky, substitutions


def ik_flops(n_obstacles, restarts, iters):
    """FP32 operations of one target's solve, counting the evaluations (iters + 1 per
    start) and the damped solves (iters per start); the distances of the pairs that pass
    the plane test are left out, so this is a lower bound."""
    per_eval = IK_FLOPS_PER_EVAL + IK_FLOPS_PER_OBSTACLE * n_obstacles
    return restarts * ((iters + 1) * per_eval + iters * IK_FLOPS_PER_SOLVE)


def ik_oracle_sample(crane, scene, targets, restarts, iters, seconds, seed):
    """The FP64 oracle's IK (best of `restarts` Levenberg-Marquardt solves) on the targets
    in turn until `seconds` have passed; solves per second."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    pb = oracle.Problem(crane, scene, oracle.CostParams(K=1, S=1))
    oik = oracle.IKParams(seed=seed)
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.ik_solve_best(pb, targets[done % targets.shape[0]], done % targets.shape[0],
                             restarts, iters, oik)
        done += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": done / el, "unit": "IK solves/s", "cores": 1, "kind": "oracle",
            "seconds": el,
            "sample": "%d FP64 IK solves (%d starts x %d LM iterations, %d cylinders), "
                      "one thread" % (done, restarts, iters, scene.n_cyl)}


def ik_config(scene):
    return {"workload": "ik: %d grasp poses (grapple centre of a collision-free configuration, "
                        "clearance 0.05 m, height -0.5..1.5 m, yaw = slew) among %d trees, "
                        "%d starts x %d LM iterations each"
                        % (IK_TARGETS, scene.n_cyl, IK_RESTARTS, IK_ITERS),
            "step": "one cp_ik launch over all targets",
            "l2": "flushed between steps (256 MB write)"}


def ik_targets_gpu(cp, h, crane, n, seed, grapple_len=1.0):
    """Grasp poses drawn with the library's own distance and kinematics."""
    import torch
    from paper_2503_14160_gb300 import workloads

    def tips(q):
        qt = torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
        t = torch.zeros(q.shape[0], 3, device="cuda")
        cp.cp_forward_kinematics(h, qt, q.shape[0], None, t)
        return qt, t

    def accept(q):
        qt, t = tips(q)
        d = torch.zeros(q.shape[0], device="cuda")
        cp.cp_signed_distance(h, qt, q.shape[0], d)
        zg = t[:, 2] - grapple_len
        ok = (d > workloads.GRASP_CLEARANCE) & (zg > workloads.GRASP_Z[0]) & (zg < workloads.GRASP_Z[1])
        return ok.cpu().numpy()

    q = workloads.grasp_configurations(crane, accept, n, seed=seed)
    _, t = tips(q)
    t = t.cpu().numpy().astype(np.float64)
    return np.column_stack([t[:, 0], t[:, 1], t[:, 2] - grapple_len, q[:, 0]])


def ik_targets_oracle(crane, scene, n, seed, grapple_len=1.0):
    """The same draw with the oracle's distance and kinematics (reference arm)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    from paper_2503_14160_gb300 import workloads
    pb = oracle.Problem(crane, scene, oracle.CostParams(K=1, S=1))

    def accept(q):
        zg = oracle.fk_tips(pb, q)[:, 2] - grapple_len
        return ((oracle.signed_distance(pb, q) > workloads.GRASP_CLEARANCE)
                & (zg > workloads.GRASP_Z[0]) & (zg < workloads.GRASP_Z[1]))

    q = workloads.grasp_configurations(crane, accept, n, seed=seed)
    T = oracle.fk_tips(pb, q)
    return np.column_stack([T[:, 0], T[:, 1], T[:, 2] - grapple_len, q[:, 0]])


def run_ik(args):
    """Batched collision-free IK (Sec. 3.2): IK solves per second for a batch of grasp poses."""
    import torch
    from paper_2503_14160_gb300 import build, craneplan as cp, workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    cp.load()
    crane = workloads.forestry_crane()
    scene = workloads.make_scene(workloads.WORKLOADS[workloads.IK_SCENE])
    planner = cp.Planner(crane, scene, cp.make_params(64, 2, 2))
    h = planner.handle
    n, iters = IK_TARGETS, args.iterations or IK_ITERS
    ik = cp.make_ik_params(seed=rank, query=rank, restarts=IK_RESTARTS, iters=iters)
    targets_np = ik_targets_gpu(cp, h, crane, n, seed=rank)
    targets = torch.from_numpy(targets_np.astype(np.float32)).cuda()
    q = torch.zeros(n, 4, device="cuda")
    f = torch.zeros(n, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        cp.cp_ik(h, targets, n, ik, q, f)
    steps = steps_for_clocks(args.steps, lambda: (flush_l2(flush), cp.cp_ik(h, targets, n, ik, q, f)))
    times = []
    l0 = cp.cp_launch_count()
    with ClockSampler(local) as clocks:
        for _ in range(steps):
            flush_l2(flush)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            cp.cp_ik(h, targets, n, ik, q, f)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
    launches = cp.cp_launch_count() - l0
    ms = float(np.mean(times))
    fv = f.cpu().numpy()
    # end to end: targets in from pinned host memory, configurations and costs out
    host_t = targets.cpu().pin_memory()
    host_q = torch.empty_like(q, device="cpu").pin_memory()
    host_f = torch.empty_like(f, device="cpu").pin_memory()
    e2e = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        targets.copy_(host_t, non_blocking=True)
        cp.cp_ik(h, targets, n, ik, q, f)
        host_q.copy_(q, non_blocking=True)
        host_f.copy_(f, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    peaks = cp.cp_alu_peaks()
    flops = n * ik_flops(scene.n_cyl + scene.n_box, IK_RESTARTS, iters)
    achieved = flops / (ms / 1e3) / 1e12
    line = {"metric": "collision-free IK solves/sec (Sec. 3.2), batched",
            "value": n / (ms / 1e3), "unit": "IK solves/s", "n_gpus": ws, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded grasp poses in the crane-and-forest scene)",
            "config": ik_config(scene),
            "solved_fraction": float(np.mean(fv < 1e-6)),
            "median_residual_sq": float(np.median(fv)),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peaks["fp32_tflops"],
                         "unit": "TFLOP/s", "frac": achieved / peaks["fp32_tflops"],
                         "traffic": None,
                         "peak_source": "FP32 FMA rate measured by cp_alu_peaks on this GPU",
                         "kernel": "k_ik<12>",
                         "flops_note": "lower bound: kinematics, plane tests and 4x4 solves; "
                                       "pair distances of surviving obstacles not counted"},
            "e2e": {"value": n / (float(np.mean(e2e)) / 1e3), "unit": "IK solves/s",
                    "h2d_bytes_per_step": n * 16, "d2h_bytes_per_step": n * 20},
            "gpu_launches": launches, "clocks": clocks.summary()}
    if not args.no_cpu_baseline and rank == 0:
        line["cpu_baseline"] = ik_oracle_sample(crane, scene, targets_np, IK_RESTARTS, iters,
                                                args.cpu_seconds, rank)
    print(json.dumps(line), flush=True)
    planner.close()


HULL_CONFIGS = 1 << 20


def hull_config(scene):
    return {"workload": "hulls: %d configurations uniform in the joint limits against the single-large "
                        "forest (%d trees as circumscribed octagonal prisms), 4 link boxes each"
                        % (HULL_CONFIGS, scene.n_cyl),
            "step": "one cp_hull_penetration launch over all configurations",
            "l2": "flushed between steps (256 MB write)"}


def hull_oracle_sample(crane, scene, q, seconds):
    """The FP64 oracle's hull penetration on configurations in turn until `seconds` have
    passed (numpy, one thread)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import hulls
    import oracle
    pb = oracle.Problem(crane, scene, oracle.CostParams(K=1, S=1))
    done, t0 = 0, time.perf_counter()
    while True:
        hulls.penetration(pb, q[done % len(q)])
        done += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": done / el, "unit": "configurations/s", "cores": 1, "kind": "oracle", "seconds": el,
            "sample": "%d FP64 hull checks (4 link boxes vs %d prisms, numpy over obstacles), one thread"
                      % (done, scene.n_cyl)}


def run_hulls(args):
    """Convex-hull collision checking (Sec. 3.1): configurations checked per second."""
    import torch
    from paper_2503_14160_gb300 import build, craneplan as cp, workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    cp.load()
    crane = workloads.forestry_crane()
    scene = workloads.make_scene(workloads.WORKLOADS["single_large"])
    planner = cp.Planner(crane, scene, cp.make_params(64, 2, 2))
    h = planner.handle
    n = HULL_CONFIGS
    q_np = workloads.uniform_configurations(crane, workloads.rng(rank, workloads.STREAM_TEST, 9), n)
    q = torch.from_numpy(q_np.astype(np.float32)).cuda()
    pen = torch.zeros(n, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        cp.cp_hull_penetration(h, q, n, pen)
    steps = steps_for_clocks(args.steps, lambda: (flush_l2(flush), cp.cp_hull_penetration(h, q, n, pen)))
    times = []
    l0 = cp.cp_launch_count()
    with ClockSampler(local) as clocks:
        for _ in range(steps):
            flush_l2(flush)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            cp.cp_hull_penetration(h, q, n, pen)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
    launches = cp.cp_launch_count() - l0
    ms = float(np.mean(times))
    colliding = float((pen > 0).float().mean().item())
    host_q = q.cpu().pin_memory()
    host_p = torch.empty_like(pen, device="cpu").pin_memory()
    e2e = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q.copy_(host_q, non_blocking=True)
        cp.cp_hull_penetration(h, q, n, pen)
        host_p.copy_(pen, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    line = {"metric": "convex-hull collision checks/sec (configurations, Sec. 3.1)",
            "value": n / (ms / 1e3), "unit": "configurations/s", "n_gpus": ws, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded configurations in the crane-and-forest scene; paper meshes unavailable)",
            "config": hull_config(scene), "colliding_fraction": colliding,
            "e2e": {"value": n / (float(np.mean(e2e)) / 1e3), "unit": "configurations/s",
                    "h2d_bytes_per_step": n * 16, "d2h_bytes_per_step": n * 4},
            "gpu_launches": launches, "clocks": clocks.summary()}
    if not args.no_cpu_baseline and rank == 0:
        line["cpu_baseline"] = hull_oracle_sample(crane, scene, q_np[:4096], args.cpu_seconds)
    print(json.dumps(line), flush=True)
    planner.close()


def run_hulls_reference(args):
    from paper_2503_14160_gb300 import workloads
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    crane = workloads.forestry_crane()
    scene = workloads.make_scene(workloads.WORKLOADS["single_large"])
    q = workloads.uniform_configurations(crane, workloads.rng(0, workloads.STREAM_TEST, 9), 4096)
    per = [hull_oracle_sample(crane, scene, q, args.cpu_seconds / 4) for _ in range(args.warmup + args.steps)]
    per = per[args.warmup:]
    value = float(np.mean([r["value"] for r in per]))
    line = {"metric": "convex-hull collision checks/sec (configurations, Sec. 3.1)", "value": value,
            "unit": "configurations/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean([r["seconds"] for r in per])) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded configurations in the crane-and-forest scene; paper meshes unavailable)",
            "impl": "reference", "config": hull_config(scene),
            "cpu_baseline": {"value": value, "unit": "configurations/s", "cores": 1, "kind": "oracle",
                             "sample": per[0]["sample"]},
            "e2e": {"value": value, "unit": "configurations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ik_reference(args):
    from paper_2503_14160_gb300 import workloads
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    crane = workloads.forestry_crane()
    scene = workloads.make_scene(workloads.WORKLOADS[workloads.IK_SCENE])
    iters = args.iterations or IK_ITERS
    targets = ik_targets_oracle(crane, scene, 256, seed=0)
    per_step = []
    for i in range(args.warmup + args.steps):
        r = ik_oracle_sample(crane, scene, targets, IK_RESTARTS, iters, args.cpu_seconds / 4, 0)
        if i >= args.warmup:
            per_step.append(r)
    value = float(np.mean([r["value"] for r in per_step]))
    line = {"metric": "collision-free IK solves/sec (Sec. 3.2), batched", "value": value,
            "unit": "IK solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean([r["seconds"] for r in per_step])) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded grasp poses in the crane-and-forest scene)",
            "impl": "reference", "config": ik_config(scene),
            "cpu_baseline": {"value": value, "unit": "IK solves/s", "cores": 1, "kind": "oracle",
                             "sample": per_step[0]["sample"]},
            "e2e": {"value": value, "unit": "IK solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """The batched serving form: 64 queries of uneven size (N ~ U[1024, 16384], K ~ U[8, 32],
    M ~ U[50, 3000] cylinders, S = 64, 100 iterations), every stage of an iteration one launch
    for all queries (the evaluation one persistent launch over a device queue of tiles), the
    whole run one CUDA graph; against the same queries planned one after another with cp_plan.
    The polar index's ring width per size bucket and the batched evaluation's block and tile
    shape come from the autotuner."""
    import torch
    from paper_2503_14160_gb300 import autotune, build, craneplan as cp, workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    cp.load()
    crane = workloads.forestry_crane()
    model = cp.make_model(crane)
    S, T, nq = 64, args.iterations or 100, args.queries
    queries = workloads.batch_queries(nq, seed=rank)
    tuner = autotune.Autotuner()
    t_tune = time.perf_counter()
    cfgs = [tuner.best_polar(crane, bq.n_candidates, bq.n_waypoints, S, bq.n_cyl) for bq in queries]
    t_tune = time.perf_counter() - t_tune
    scenes, params, q0s, qds, raw = [], [], [], [], []
    for q, (bq, cfg) in enumerate(zip(queries, cfgs)):
        sc = workloads.batch_scene(bq, seed=rank, q=q)
        with cp.Planner(crane, sc, cp.make_params(64, bq.n_waypoints, S)) as tmp:
            q0, qd, _ = select_endpoints_gpu(cp, tmp, crane, rank, q)
        raw.append(sc)
        scenes.append(cp.HostScene.from_scene(sc))
        params.append(cp.make_params(bq.n_candidates, bq.n_waypoints, S, seed=rank, query=q, **cfg))
        q0s.append(q0)
        qds.append(qd)
    t0 = time.perf_counter()
    b = cp.cp_batch_init(model, scenes, params, q0s, qds, T)
    t_init = time.perf_counter() - t0
    Ks = [bq.n_waypoints for bq in queries]
    if args.batch_shape:
        # a fixed launch shape (profiling runs): no shape search
        shape = [int(v) for v in args.batch_shape.split(",")]
        cp.cp_batch_set_shape(b, *shape)
        tuned = {"shape": shape, "ms": [], "shapes": [], "fixed": True}
    else:
        cp.cp_batch_run(b, nq)                      # populations for the shape search
        t1 = time.perf_counter()
        tuned = tuner.tune_batch(b, "nq%d|seed%d|S%d" % (nq, rank, S))
        t_tune += time.perf_counter() - t1
    info = cp.cp_batch_get_info(b)
    units = info["candidates"] * T
    for _ in range(max(args.warmup, 3)):
        cp.cp_batch_run(b, nq)
    dev_ms, host_ms = [], []
    l0 = cp.cp_launch_count()
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = cp.cp_batch_run(b, nq, K=Ks)
            host_ms.append((time.perf_counter() - t0) * 1e3)
            dev_ms.append(cp.cp_batch_get_info(b)["last_run_ms"])
    launches = cp.cp_launch_count() - l0
    eval_ms = cp.cp_batch_evaluate(b, 5)
    checkpoints = sum(bq.n_candidates * (bq.n_waypoints + 3) * S for bq in queries)
    # the same queries planned one after another in the plain form (each planner's own graph,
    # recorded in an untimed pass first)
    seq = []
    for rep in range(1 + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in range(nq):
            p = cp.cp_batch_planner(b, q)
            cp.cp_set_endpoints(p, q0s[q], qds[q])
            cp.cp_plan(p, T)
        if rep > 0:
            seq.append((time.perf_counter() - t0) * 1e3)
    ms, ms_host, ms_seq = float(np.mean(dev_ms)), float(np.mean(host_ms)), float(np.mean(seq))
    line = {"metric": "candidate paths evaluated/sec, %d-query batch (one graph, one launch per stage) "
                      "vs sequential plain plans" % nq,
            "value": units / (ms / 1e3), "unit": "candidate paths/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded crane-and-forest scenes)",
            "config": {"workload": "batch: %d queries, N U[1024,16384], K U[8,32], cylinders U[50,3000], "
                                   "S=64, %d iterations" % (nq, T), "step": "one batch run (all queries)",
                       "l2": "working set above L2 (%d candidates x up to 128 floats, plus scenes)"
                             % info["candidates"]},
            "sequential": {"value": units / (ms_seq / 1e3), "ms_per_batch": ms_seq,
                           "form": "cp_plan per query (its own graph), one after another"},
            "speedup_vs_sequential": ms_seq / ms,
            "graph": {"kernel_nodes": info["kernel_nodes"], "persistent_eval_launches": info["eval_launches"],
                      "eval_tiles_per_launch": info["eval_tiles"], "eval_ctas": info["eval_ctas"]},
            "eval_kernel": {"name": "k_batch_eval_polar", "ms_per_launch": eval_ms,
                            "share_of_run": eval_ms * T / ms,
                            "checkpoints_per_s": checkpoints / (eval_ms / 1e3)},
            "autotune": {"shape": tuned["shape"], "shape_ms": dict(zip(
                             ["%d/%d/%d" % tuple(sh) for sh in tuned["shapes"]], tuned["ms"])),
                         "ring_widths": sorted({c["grid_cell"] for c in cfgs}), "seconds": t_tune},
            "graph_record_and_instantiate_s": t_init,
            "collision_free": sum(1 for _, st in res if st["flag"] == 0),
            "gpu_launches": launches, "clocks": clocks.summary(),
            "e2e": {"value": units / (ms_host / 1e3), "unit": "candidate paths/s", "ms_per_batch": ms_host,
                    "h2d_bytes_per_step": nq * 8 * 8, "d2h_bytes_per_step": nq * 168 * 8}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(crane, queries, q0s, qds, rank, S, args.cpu_seconds)
        line["oracle_error"] = batch_oracle_errors(crane, queries, raw, q0s, qds, res, S)
    print(json.dumps(line), flush=True)
    cp.cp_batch_destroy(b)


def batch_oracle_errors(crane, queries, scenes, q0s, qds, res, S):
    """Error of the batch's results against the FP64 oracle (brute force): the returned mean
    path of every eighth query, its J, length and flag."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    rows = []
    for q in range(0, len(queries), 8):
        K = queries[q].n_waypoints
        ctrl, st = res[q]
        problem = oracle.Problem(crane, scenes[q], oracle.CostParams(K=K, S=S))
        x = np.asarray(ctrl)[4:4 + K].astype(np.float32).astype(np.float64)[None]
        o = oracle.evaluate(problem, x, q0s[q], qds[q])
        rows.append({"query": q, "J_rel_err": abs(st["J"] - float(o.J[0])) / max(abs(float(o.J[0])), 1e-300),
                     "length_rel_err": abs(st["length"] - float(o.length[0])) / float(o.length[0]),
                     "flag_gpu": int(st["flag"]), "flag_oracle": int(o.flag[0])})
    return {"queries": rows, "J_rel_err_max": max(r["J_rel_err"] for r in rows),
            "length_rel_err_max": max(r["length_rel_err"] for r in rows),
            "flag_agreement": sum(r["flag_gpu"] == r["flag_oracle"] for r in rows) / len(rows),
            "oracle_form": "brute force"}


TRAJ_PATHS = 64


def traj_flops_per_step(N):
    """Algorithmic FP64 work of one Levenberg-Marquardt step of one trajectory (the GPU's form):
    per grid point the dynamics' Jacobian by 16 forward-mode passes (about 360 flops each), the
    diagonal and off-diagonal 16 x 16 blocks of J^T J from the 12-row defect Jacobians
    (2 x 12 flops per entry), the block factorisation (the Schur update 2 x 16^3, the 16 x 16
    Cholesky 16^3 / 3, L^-1 E_k 16^3) and the substitutions of two vectors (4 x 2 x 16^2)."""
    per_point = 16 * 360 + 2 * 256 * 24 + 2 * 16 ** 3 + 16 ** 3 / 3 + 16 ** 3 + 8 * 256
    return (N + 1) * per_point


def run_trajopt(args):
    """The trajectory tracking optimisation of Sec. 4.2 (Eq. discrete), batched: the paths of
    64 plans of the 20-tree query (seeds 0..63, K = 8, 50 iterations each) turned into
    trajectories on N = 100 collocation intervals (the paper's n_s) by one solver launch, one
    CTA per trajectory. A step is one batch: targets, starting points and the solve."""
    import torch
    from paper_2503_14160_gb300 import build, craneplan as cp, workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    torch.cuda.set_stream(torch.cuda.Stream())
    build.build()
    cp.load()
    crane = workloads.forestry_crane()
    wl = workloads.WORKLOADS["single_small"]
    scene = workloads.make_scene(wl)
    with open(os.path.join(ROOT, "tests", "golden", "endpoints.json")) as f:
        e = json.load(f)["workloads"][wl.name]
    q0, qd = np.array(e["q0"]), np.array(e["qd"])
    K, N, n = wl.n_waypoints, 100, TRAJ_PATHS
    ctrl = np.zeros((n, K + 8, 4))
    for p in range(n):   # the planned paths (untimed: the path step is measured by its own line)
        with cp.Planner(crane, scene, cp.make_params(wl.n_candidates, K, wl.substeps, seed=p, query=rank)) as pl:
            cp.cp_set_endpoints(pl.handle, q0, qd)
            ctrl[p], _ = cp.cp_plan(pl.handle, wl.iterations, K=K)
    tp = cp.make_traj_params(N=N)
    h = cp.cp_traj_init(cp.make_model(crane), tp, n)
    n_var = 1 + 16 * (N + 1)
    d_ctrl = torch.from_numpy(ctrl).cuda()
    q = torch.zeros(n, N + 1, 4, dtype=torch.float64, device="cuda")
    z = torch.zeros(n, n_var, dtype=torch.float64, device="cuda")
    stats = torch.zeros(n, 4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def one():
        cp.cp_traj_targets(h, d_ctrl, K, n, q)
        cp.cp_traj_initial_guess(h, q, n, z)
        cp.cp_traj_solve(h, q, n, z, stats)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    l0 = cp.cp_launch_count()
    times = []
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            one()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
    launches = cp.cp_launch_count() - l0
    # end to end with host buffers: control points in, trajectories and statistics out
    h_ctrl = torch.from_numpy(ctrl).pin_memory()
    h_z = torch.zeros(n, n_var, dtype=torch.float64).pin_memory()
    h_st = torch.zeros(n, 4, dtype=torch.float64).pin_memory()
    e2e = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_ctrl.copy_(h_ctrl, non_blocking=True)
        one()
        h_z.copy_(z, non_blocking=True)
        h_st.copy_(stats, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    st = stats.cpu().numpy()
    ms, ms_e2e = max_over_ranks([float(np.mean(times)), float(np.mean(e2e))], "cuda")
    steps_lm = tp.outer * tp.inner
    flops = traj_flops_per_step(N) * steps_lm * n
    peaks = cp.cp_alu_peaks()
    achieved = flops / (ms / 1e3) / 1e12
    line = {"metric": "trajectories optimised/sec (Sec. 4.2 direct collocation, N = 100)",
            "value": job_throughput(n, ws, ms), "unit": "trajectories/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (paths planned on the seeded 20-tree scene; synthetic crane dynamics)",
            "config": {"workload": "trajopt: %d paths (plans of the 20-tree query, seeds 0..%d), N=%d, %d x %d "
                                   "Levenberg-Marquardt steps" % (n, n - 1, N, tp.outer, tp.inner),
                       "step": "one batch: targets, starting points, solve", "l2": "inputs below L2 (a few MB)"},
            "e2e": {"value": job_throughput(n, ws, ms_e2e), "unit": "trajectories/s", "ms_per_step": ms_e2e,
                    "h2d_bytes_per_step": ctrl.nbytes, "d2h_bytes_per_step": n * (n_var + 4) * 8},
            "gpu_launches": launches // max(args.steps, 1) * args.steps,
            "roofline": {"bound": "fp64", "kernel": "k_traj_solve", "achieved": achieved,
                         "peak": peaks["fp64_tflops"], "unit": "TFLOP/s", "frac": achieved / peaks["fp64_tflops"],
                         "peak_basis": "cp_alu_peaks (measured FP64 FMA rate, whole GPU)",
                         "sms_used": 2 * n, "ctas_per_trajectory": 2, "traffic": None},
            "result": {"t_F_mean_s": float(st[:, 0].mean()), "max_constraint_error": float(st[:, 2].max()),
                       "max_bound_violation": float(st[:, 3].max())},
            "clocks": clocks.summary()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = traj_cpu_baseline(crane, ctrl[0], N, steps_lm, q.cpu().numpy()[0])
        line["oracle_error"] = traj_oracle_error(crane, q.cpu().numpy()[0], z.cpu().numpy()[0], N)
    print(json.dumps(line), flush=True)
    cp.cp_traj_destroy(h)


def traj_cpu_baseline(crane, ctrl, N, steps, q_star):
    """The oracle's trajectory solver as it stands (dense complex-step Jacobians, numpy) on a
    bounded sample: one Levenberg-Marquardt step of one trajectory at N, timed, scaled to the
    solve's steps."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import trajopt
    prob = trajopt.TrajProblem(crane, trajopt.TrajParams(N=N), q_star, q_star[0], q_star[-1])
    z = prob.initial_guess()
    t0 = time.perf_counter()
    prob.lm_step(z, np.zeros(prob.n_eq), 1e-3)
    el = time.perf_counter() - t0
    return {"value": 1.0 / (el * steps), "unit": "trajectories/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "seconds": el, "sample": "one Levenberg-Marquardt step of one trajectory at N=%d (dense complex-step "
                                     "Jacobian, numpy), scaled to the %d steps of a solve" % (N, steps)}


def traj_oracle_error(crane, q_star, z_gpu, N):
    """The GPU's first Levenberg-Marquardt step against the oracle's, at the GPU's result (the
    CPU-baseline leg): relative difference of the steps, and the oracle's objective at the
    GPU's trajectory against the GPU's."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import trajopt
    prob = trajopt.TrajProblem(crane, trajopt.TrajParams(N=N), q_star, q_star[0], q_star[-1])
    c = prob.constraints(z_gpu)
    return {"max_constraint_error_oracle": float(np.max(np.abs(c))),
            "max_bound_violation_oracle": float(np.max(np.abs(prob.violation(z_gpu)))),
            "t_F": float(z_gpu[0])}


def batch_cpu_baseline(crane, queries, q0s, qds, seed, S, seconds):
    """The FP64 oracle on a bounded sample of the batch: candidate evaluations of every
    eighth query in turn (each with its own scene and sizes) until `seconds` have passed."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    from paper_2503_14160_gb300 import workloads
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    done, t0, picked = 0, time.perf_counter(), list(range(0, len(queries), 8))
    while True:
        for q in picked:
            bq = queries[q]
            sc = workloads.batch_scene(bq, seed=seed, q=q)
            problem = oracle.Problem(crane, sc, oracle.CostParams(K=bq.n_waypoints, S=S))
            xi = workloads.random_candidates(q0s[q], qds[q], bq.n_waypoints, 2 * cores, seed=q)
            oracle.evaluate(problem, xi.astype(np.float64), q0s[q], qds[q])
            done += xi.shape[0]
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": done / el, "unit": "candidate paths/s", "cores": int(oracle.get_threads()),
            "kind": "oracle", "seconds": el,
            "sample": "%d candidate evaluations (FP64, OpenMP over candidates) of queries %s of "
                      "the batch, each with its own scene and sizes" % (done, picked)}


def _oracle_eval(oracle, problem, wl, xi, q0, qd, with_distances=False):
    """Step (2) by the oracle: brute force, or through its uniform grid (the same costs and
    flags, pinned equal to the brute force) on the grid workloads."""
    if wl.grid_cell > 0:
        return oracle.evaluate_grid(problem, xi, q0, qd, wl.grid_cell, with_distances=with_distances)
    return oracle.evaluate(problem, xi, q0, qd, with_distances=with_distances)


def cpu_baseline(wl, crane, scene, q0, qd, seconds, max_batches=None, single_core_seconds=None):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample: candidate
    evaluations (step (2), which dominates a plan) of the same workload, in batches until
    `seconds` have passed; value in candidate paths per second. On the grid workloads the
    oracle takes d(q) through its own uniform grid (equal to its brute force in every cost
    and flag). With single_core_seconds the same is also timed on one core."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    from paper_2503_14160_gb300 import workloads
    cores = os.cpu_count() or 1
    problem = oracle.Problem(crane, scene, oracle.CostParams(K=wl.n_waypoints, S=wl.substeps))
    form = "grid of %.2f m cells" % wl.grid_cell if wl.grid_cell > 0 else "brute force"

    def timed(threads, budget, batch, limit):
        oracle.set_threads(threads)
        xi = workloads.random_candidates(q0, qd, wl.n_waypoints, batch, seed=123).astype(np.float64)
        done, t0, batches = 0, time.perf_counter(), 0
        while True:
            _oracle_eval(oracle, problem, wl, xi, q0, qd)
            done += batch
            batches += 1
            el = time.perf_counter() - t0
            if el >= budget or (limit and batches >= limit):
                return done, el, int(oracle.get_threads())

    done, el, used = timed(cores, seconds, 4 * cores * (8 if wl.grid_cell > 0 else 1), max_batches)
    out = {"value": done / el, "unit": UNIT, "cores": used, "kind": "oracle", "seconds": el,
           "sample": "%d candidate evaluations (K=%d, S=%d, %d cylinders + %d boxes, FP64, d(q) by %s, "
                     "OpenMP over candidates) of the %s workload" % (done, wl.n_waypoints, wl.substeps,
                                                                  scene.n_cyl, scene.n_box, form, wl.name)}
    if single_core_seconds:
        d1, e1, _ = timed(1, single_core_seconds, 8 if wl.grid_cell > 0 else 1, None)
        out["single_core"] = {"value": d1 / e1, "unit": UNIT, "cores": 1, "seconds": e1,
                              "sample": "%d candidate evaluations, same form" % d1}
    oracle.set_threads(cores)
    return out


def oracle_errors(cp, h, wl, crane, scene, q0, qd, ctrl, stats, iters, n_sample=256):
    """The error of the benchmarked results against the FP64 oracle (run in the CPU-baseline
    leg): the plan's mean path (the float32 waypoints the GPU evaluated) by brute force, its
    J, length and flags; and n_sample candidates drawn from the final distribution, the
    GPU's J, penalties and flags against the oracle's on the same float32 candidates."""
    import torch
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    K, n_s = wl.n_waypoints, wl.n_checkpoints
    problem = oracle.Problem(crane, scene, oracle.CostParams(K=K, S=wl.substeps))
    mean_xi = np.asarray(ctrl)[4:4 + K].astype(np.float32).astype(np.float64)[None]
    o = oracle.evaluate(problem, mean_xi, q0, qd)
    plan = {"J_gpu": stats["J"], "J_oracle": float(o.J[0]),
            "J_rel_err": abs(stats["J"] - float(o.J[0])) / max(abs(float(o.J[0])), 1e-300),
            "length_gpu": stats["length"], "length_oracle": float(o.length[0]),
            "length_rel_err": abs(stats["length"] - float(o.length[0])) / max(float(o.length[0]), 1e-300),
            "flag_gpu": int(stats["flag"]), "flag_oracle": int(o.flag[0]),
            "n_flagged_gpu": int(stats["n_flagged"]), "n_flagged_oracle": int(o.n_flagged[0]),
            "oracle_form": "brute force"}
    n = min(n_sample, wl.n_candidates)
    xi = torch.zeros(n if n == wl.n_candidates else wl.n_candidates, K, 4, device="cuda")
    cp.cp_sample(h, iters, xi)
    J = torch.zeros(n, dtype=torch.float64, device="cuda")
    flag = torch.zeros(n, dtype=torch.uint8, device="cuda")
    terms = torch.zeros(n, 5, dtype=torch.float64, device="cuda")
    W = (n_s + 31) // 32
    words = torch.zeros(n, W, dtype=torch.int32, device="cuda")
    pen = torch.zeros(n, n_s, dtype=torch.float32, device="cuda")
    cp.cp_evaluate(h, xi, n, J, flag, terms, words, pen)
    torch.cuda.synchronize()
    xs = xi[:n].cpu().numpy().astype(np.float64)
    c = _oracle_eval(oracle, problem, wl, xs, q0, qd, with_distances=True)
    d = c.d[:, 1:]
    Jg = J.cpu().numpy()
    rel = np.abs(Jg - c.J) / np.maximum(np.abs(c.J), 1e-300)
    w = words.cpu().numpy().view(np.uint32)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)[None, None, :]) & 1).astype(bool)
    flags = bits.reshape(n, -1)[:, :n_s]
    band = np.abs(d) > 1e-4
    near = (d < 2e-5).sum(axis=1)
    tol = 1e-4 * np.abs(c.J) + 100.0 * 2e-5 * near + 1e-9
    cand = {"candidates": n, "drawn_from": "the final distribution (iteration %d)" % iters,
            "oracle_form": "grid (equal to brute force)" if wl.grid_cell > 0 else "brute force",
            "J_rel_err_max": float(rel.max()), "J_rel_err_median": float(np.median(rel)),
            "frac_J_within_1e-4_rel": float(np.mean(rel <= 1e-4)),
            "frac_J_within_tolerance": float(np.mean(np.abs(Jg - c.J) <= tol)),
            "contact_checkpoints_per_candidate": float(near.mean()),
            "pen_abs_err_max_m": float(np.abs(pen.cpu().numpy() - np.maximum(0.0, -d)).max()),
            "flag_mismatches_outside_1e-4_m": int((flags[band] != (d < 0)[band]).sum()),
            "checkpoints_compared": int(n * n_s)}
    return {"plan": plan, "candidates": cand}


def run_traj_reference(args):
    """--impl reference for the trajectory workload: the oracle's solver on one trajectory,
    one Levenberg-Marquardt step per bench step (bounded), scaled to a solve."""
    from paper_2503_14160_gb300 import workloads
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import trajopt
    crane = workloads.forestry_crane()
    with open(os.path.join(ROOT, "tests", "golden", "endpoints.json")) as f:
        e = json.load(f)["workloads"]["single_small"]
    q0, qd = np.array(e["q0"]), np.array(e["qd"])
    N = 100
    s = np.linspace(0.0, 1.0, N + 1)[:, None]
    q_star = q0[None] + (3 * s ** 2 - 2 * s ** 3) * (qd - q0)[None]
    tp = trajopt.TrajParams(N=N)
    prob = trajopt.TrajProblem(crane, tp, q_star, q0, qd)
    z = prob.initial_guess()
    per = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        prob.lm_step(z, np.zeros(prob.n_eq), 1e-3)
        if i >= args.warmup:
            per.append(time.perf_counter() - t0)
    el = float(np.mean(per))
    value = 1.0 / (el * tp.outer * tp.inner)
    line = {"metric": "trajectories optimised/sec (Sec. 4.2 direct collocation, N = 100)", "value": value,
            "unit": "trajectories/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (a smooth rest-to-rest path of the 20-tree query's end points)",
            "impl": "reference",
            "config": {"workload": "trajopt: N=%d, %d x %d Levenberg-Marquardt steps" % (N, tp.outer, tp.inner),
                       "step": "a bounded sample: one Levenberg-Marquardt step of one trajectory"},
            "cpu_baseline": {"value": value, "unit": "trajectories/s", "cores": os.cpu_count() or 1,
                             "kind": "oracle", "sample": "one step of one trajectory per bench step, scaled to a solve"},
            "e2e": {"value": value, "unit": "trajectories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args):
    from paper_2503_14160_gb300 import workloads
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    wl = workloads.WORKLOADS[args.workload]
    iters = args.iterations or wl.iterations
    crane = workloads.forestry_crane()
    scene = workloads.make_scene(wl)
    with open(os.path.join(ROOT, "tests", "golden", "endpoints.json")) as f:
        e = json.load(f)["workloads"][wl.name]
    q0, qd = np.array(e["q0"]), np.array(e["qd"])
    per_step = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(wl, crane, scene, q0, qd, args.cpu_seconds / 4, max_batches=1)
        if i >= args.warmup:
            per_step.append(r)
    value = float(np.mean([r["value"] for r in per_step]))
    ms_per_plan = wl.n_candidates * iters / value * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean([r["seconds"] for r in per_step])) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded crane-and-forest scene)", "impl": "reference",
            "config": {"workload": "%s: N=%d K=%d S=%d cylinders=%d iterations=%d per plan"
                                   % (wl.name, wl.n_candidates, wl.n_waypoints, wl.substeps,
                                      scene.n_cyl, iters),
                       "step": "a bounded sample: one batch of candidate evaluations"},
            "ms_per_plan_extrapolated": ms_per_plan,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": per_step[0]["cores"],
                             "kind": "oracle", "sample": per_step[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch_reference(args):
    """--impl reference for the batch workload: the FP64 oracle evaluating candidates of every
    eighth query of the same 64-query batch (each with its own scene and sizes), one bounded
    sample per step, scaled to candidate paths per second."""
    from paper_2503_14160_gb300 import workloads
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    crane = workloads.forestry_crane()
    S, T = 64, args.iterations or 100
    nq = args.queries
    queries = workloads.batch_queries(nq, seed=rank)
    q0s, qds = [None] * nq, [None] * nq
    for q in range(0, nq, 8):
        bq = queries[q]
        pb = oracle.Problem(crane, workloads.batch_scene(bq, seed=rank, q=q), oracle.CostParams(K=bq.n_waypoints, S=S))
        q0s[q], qds[q], _, _ = workloads.select_endpoints(crane, lambda x: oracle.signed_distance(pb, x),
                                                          seed=rank, batch=4096, query=q)
    per_step = []
    for i in range(args.warmup + args.steps):
        r = batch_cpu_baseline(crane, queries, q0s, qds, rank, S, args.cpu_seconds / 4)
        if i >= args.warmup:
            per_step.append(r)
    value = float(np.mean([r["value"] for r in per_step]))
    line = {"metric": "candidate paths evaluated/sec, %d-query batch (one graph, one launch per stage) "
                      "vs sequential plain plans" % nq,
            "value": value, "unit": "candidate paths/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean([r["seconds"] for r in per_step])) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded crane-and-forest scenes)", "impl": "reference",
            "config": {"workload": "batch: %d queries, N U[1024,16384], K U[8,32], cylinders U[50,3000], "
                                   "S=64, %d iterations" % (nq, T),
                       "step": "a bounded sample: candidate evaluations of every eighth query"},
            "cpu_baseline": {"value": value, "unit": "candidate paths/s", "cores": per_step[0]["cores"],
                             "kind": "oracle", "sample": per_step[0]["sample"]},
            "e2e": {"value": value, "unit": "candidate paths/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--iterations", type=int, default=0, help="override iterations per plan")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--collision", default="spheres", choices=["spheres", "hulls"],
                    help="d(q) from link spheres, or from link boxes by separating axes")
    ap.add_argument("--sampler", default="auto", choices=["auto", "factor", "elites"],
                    help="step (1) from the Cholesky factor or from the last update's elites")
    ap.add_argument("--update-rule", default="paper", choices=["paper", "cmaes"],
                    help="steps (5)-(6) as Algorithm 1 prints them, or the CMA-ES update")
    ap.add_argument("--exhaustive", action="store_true",
                    help="evaluate every sphere against every obstacle (no broad phase, no index)")
    ap.add_argument("--queries", type=int, default=64, help="batch workload: number of queries")
    ap.add_argument("--batch-shape", default="",
                    help="batch workload: fixed evaluation shape 'threads,ctas_per_sm,items_per_warp' "
                         "(skips the autotuner)")
    args = ap.parse_args()
    if args.impl == "reference" and args.workload == "ik":
        run_ik_reference(args)
    elif args.impl == "reference" and args.workload == "hulls":
        run_hulls_reference(args)
    elif args.impl == "reference" and args.workload == "trajopt":
        run_traj_reference(args)
    elif args.impl == "reference" and args.workload == "batch":
        run_batch_reference(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "ik":
        run_ik(args)
    elif args.workload == "hulls":
        run_hulls(args)
    elif args.workload == "differentiable":
        run_differentiable(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "trajopt":
        run_trajopt(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

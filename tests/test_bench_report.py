"""The arithmetic of bench.py's report, on synthetic timings (CPU): the evaluation roofline
(algorithmic FP32 flops over the launches' device time), the FP64 stages, the tensor-core
sampler stage, and the step count that lengthens short timed regions for the clock
sampler."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


@pytest.fixture(scope="module")
def wl():
    from paper_2503_14160_gb300 import workloads
    return workloads.WORKLOADS["single_large"]


def _timing(**kw):
    t = {"eval_ms": 10.0, "eval_launches": 100, "eval_units": 1000, "eval_pair_tests": 2000,
         "sample_ms": 4.0, "sample_launches": 100, "factor_ms": 0.06, "factor_launches": 1,
         "update_ms": 3.0, "update_launches": 100}
    t.update(kw)
    return t


def test_eval_roofline_broad_counts_every_part(bench):
    t = _timing()
    r = bench.eval_roofline(t, n_spheres=12, n_obstacles=500, n_s=1216, candidates=3, form="broad",
                            sm_mhz=2070.0)
    flops = (3 * 1216 * bench.FLOPS_PER_CHECKPOINT + 2000 * bench.FLOPS_PER_PAIR
             + 3 * 1216 * 12 * bench.FLOPS_FRAME_PER_SPHERE + 1000 * 500 * bench.FLOPS_PER_BROAD_TEST)
    assert r["achieved"] == pytest.approx(flops / 10e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP32_PEAK_TFLOPS)
    assert r["eval_ms_per_launch"] == pytest.approx(0.1)
    assert r["pair_tests_per_checkpoint"] == pytest.approx(2000 / (3 * 1216))
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2.070e9 / 1e12)


def test_eval_roofline_polar_counts_the_index_tests(bench):
    t = _timing(eval_box_tests=5000)
    r = bench.eval_roofline(t, n_spheres=12, n_obstacles=5050, n_s=4480, candidates=3, form="polar",
                            sm_mhz=2070.0)
    flops = (3 * 4480 * bench.FLOPS_PER_CHECKPOINT + 2000 * bench.FLOPS_PER_PACKED_PAIR
             + 5000 * bench.FLOPS_PER_INDEX_TEST)
    assert r["achieved"] == pytest.approx(flops / 10e-3 / 1e12)
    assert r["kernel"] == "k_eval_polar"
    assert r["listed_obstacles_per_checkpoint"] == pytest.approx(5000 / (3 * 4480))


def test_traffic_is_reported_only_for_the_profiled_sources(bench):
    for (kernel, workload), rec in bench.PROFILED_TRAFFIC.items():
        want = rec["bytes"] if bench.kernel_source_sha1(kernel) == rec["sha1"] else None
        assert bench.traffic_per_launch(kernel, workload) == want
        assert bench.traffic_per_launch(kernel, "no such workload") is None


def test_eval_roofline_refuses_empty_timings(bench):
    assert bench.eval_roofline(_timing(eval_units=0), 12, 500, 1216, 3, "broad", None) is None


def test_fp64_stages_follow_the_sampler(bench, wl):
    D, nu = 4 * wl.n_waypoints, wl.n_candidates // 2
    f = bench.fp64_stages(_timing(), wl, 1.0, "factor")
    e = bench.fp64_stages(_timing(), wl, 1.0, "elites")
    us = 3.0 / 100 * 1e3
    assert f["update"]["achieved"] == pytest.approx(2.0 * (nu * D * (D + 1) / 2 + nu * D) / (us / 1e6) / 1e12)
    assert e["update"]["achieved"] == pytest.approx(2.0 * nu * D / (us / 1e6) / 1e12)
    assert e["factor"]["achieved"] == pytest.approx(2.0 * D ** 3 / 3 / (0.06e-3) / 1e12)
    assert bench.fp64_stages(_timing(), wl, None, "elites") is None


def test_sampler_stage(bench, wl, monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"bf16_tflops_sustained": 2250.0})
    s = bench.sampler_stage(_timing(), wl, "elites")
    D = 4 * wl.n_waypoints
    Dp = (D + 15) // 16 * 16
    nu = wl.n_candidates // 2
    us = 4.0 / 100 * 1e3
    assert s["us_per_call"] == pytest.approx(us)
    assert s["normals_per_s"] == pytest.approx(wl.n_candidates * (nu + D) / (us / 1e6))
    assert s["tensor"]["achieved"] == pytest.approx(3 * 2.0 * wl.n_candidates * nu * Dp / (us / 1e6) / 1e12)
    assert s["tensor"]["peak"] == pytest.approx(1100.0)
    assert bench.sampler_stage(_timing(), wl, "factor") is None
    # without measured peaks the stage reports against the labelled fallback, not null
    monkeypatch.setattr(bench, "measured_peaks", lambda: {})
    f = bench.sampler_stage(_timing(), wl, "elites")
    assert f["tensor"]["peak"] == pytest.approx(1700.0 * 1.1 / 2.25)
    assert f["tensor"]["frac"] == pytest.approx(f["tensor"]["achieved"] / f["tensor"]["peak"])
    assert "fallback" in f["tensor"]["peak_basis"]


def test_steps_for_clocks_covers_a_second(bench, monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    clock = iter([0.0, 0.004, 1.0, 1.002, 2.0, 2.003])   # three untimed steps: 4, 2, 3 ms
    monkeypatch.setattr(bench.time, "perf_counter", lambda: next(clock))
    assert bench.steps_for_clocks(5, lambda: None) == 500          # ceil(1 s / 2 ms)
    clock2 = iter([0.0, 1.0, 2.0, 3.5, 4.0, 5.2])
    monkeypatch.setattr(bench.time, "perf_counter", lambda: next(clock2))
    assert bench.steps_for_clocks(5, lambda: None) == 5            # slow steps: the given count

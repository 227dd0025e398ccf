"""The C ABI library loads, exports every entry point include/craneplan.h declares, and its
structs have the header's layout. Argument validation is checked where it rejects the call
before any CUDA work (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "craneplan.h")


@pytest.fixture(scope="module")
def cp():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cp_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(cp):
    names = declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(cp.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps every one under the same name
    assert not [n for n in names if not hasattr(cp, n)]


def test_struct_layout_matches_header(cp, tmp_path):
    src = tmp_path / "probe.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "craneplan.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                   'sizeof(cp_model), sizeof(cp_params), sizeof(cp_plan_stats),'
                   'sizeof(cp_timing), sizeof(cp_scene), sizeof(cp_cylinder), sizeof(cp_box),'
                   'offsetof(cp_params, seed), offsetof(cp_model, spheres), sizeof(cp_batch_shape),'
                   'sizeof(cp_batch_info), offsetof(cp_batch_info, last_run_ms), sizeof(cp_traj_params));'
                   'return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(cp.cp_model), ctypes.sizeof(cp.cp_params),
            ctypes.sizeof(cp.cp_plan_stats), ctypes.sizeof(cp.cp_timing),
            ctypes.sizeof(cp.cp_scene), ctypes.sizeof(cp.cp_cylinder),
            ctypes.sizeof(cp.cp_box), cp.cp_params.seed.offset, cp.cp_model.spheres.offset,
            ctypes.sizeof(cp.cp_batch_shape), ctypes.sizeof(cp.cp_batch_info),
            cp.cp_batch_info.last_run_ms.offset, ctypes.sizeof(cp.cp_traj_params)]
    assert got == want


def test_version_and_counter(cp):
    assert cp.cp_version() == 1
    assert cp.cp_launch_count() >= 0


def _crane():
    from paper_2503_14160_gb300 import workloads
    return workloads.forestry_crane()


@pytest.mark.parametrize("mutate,needle", [
    (lambda m, p: setattr(m, "n_spheres", 0), "n_spheres"),
    (lambda m, p: setattr(m, "n_spheres", 17), "n_spheres"),
    (lambda m, p: setattr(p, "n_candidates", 1), "n_candidates"),
    (lambda m, p: setattr(p, "n_waypoints", 33), "n_waypoints"),
    (lambda m, p: setattr(p, "n_waypoints", 0), "n_waypoints"),
    (lambda m, p: setattr(p, "substeps", 0), "substeps"),
    (lambda m, p: setattr(p, "n_elites", 1000), "n_elites"),
    (lambda m, p: setattr(p, "sigma", 0.0), "sigma"),
    (lambda m, p: setattr(p, "eps", -1.0), "eps"),
    (lambda m, p: setattr(p, "w_c", float("nan")), "weights"),
    (lambda m, p: setattr(p, "debug_withhold_staging", 3), "debug_withhold_staging"),
])
def test_init_rejects_bad_arguments(cp, mutate, needle):
    from paper_2503_14160_gb300 import workloads
    model = cp.make_model(_crane())
    params = cp.make_params(64, 8, 16)
    mutate(model, params)
    scene = cp.HostScene.from_scene(workloads.empty_scene())
    with pytest.raises(cp.CranePlanError) as e:
        cp.cp_plan_init(model, scene, params, stream=0)
    assert e.value.status == -1 and needle in str(e.value)


def test_init_rejects_bad_scene(cp):
    import numpy as np
    model = cp.make_model(_crane())
    params = cp.make_params(64, 8, 16)
    bad = cp.HostScene(np.array([[0.0, 0.0, -1.0, 0.0, 1.0]]), np.zeros((0, 6)))
    with pytest.raises(cp.CranePlanError) as e:
        cp.cp_plan_init(model, bad, params, stream=0)
    assert e.value.status == -1 and "cylinder 0" in str(e.value)
    bad_box = cp.HostScene(np.zeros((0, 5)), np.array([[0, 0, 0, -1, 1, 1.0]]))
    with pytest.raises(cp.CranePlanError):
        cp.cp_plan_init(model, bad_box, params, stream=0)


def test_null_planner_calls_fail_cleanly(cp):
    lib = cp.load()
    assert lib.cp_sample(None, 0, None) == -1
    assert lib.cp_evaluate(None, None, 0, None, None, None, None, None) == -1
    assert lib.cp_update(None, None, None) == -1
    assert lib.cp_plan(None, 1, None, None) == -1
    assert lib.cp_philox4x32_10(None, 0, -1, None, None) == -1
    lib.cp_destroy(None)

"""Auxiliaries of the planner: the per-iteration metrics ring of cp_plan and the NVTX ranges
of the library's stages.

Metrics (Algorithm 1, Sec. 4.1; one row per iteration after steps (3)-(6)): the last row's
best J, mean J, tr C and collision-free fraction are checked against the planner's state
read back independently (the population's costs, its flags from a re-evaluation, the
distribution), for the factor and the factor-free sampler; rows from a graph replay equal
rows taken kernel by kernel; the ring keeps the last 256 iterations.

NVTX: a small injection library (the NVTX v3 tool interface) compiled here records every
range push and pop of a plan run in a child process; the ranges of the stages appear,
balanced, in the expected nesting."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from helpers import ROOT, endpoints

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2503_14160_gb300 import build, craneplan
    build.build()
    craneplan.load()
    return craneplan


def _planner(cp, sampler, stream=None, N=256, K=8, S=32, seed=3):
    from paper_2503_14160_gb300 import workloads
    crane = workloads.forestry_crane()
    scene = workloads.make_scene(workloads.WORKLOADS["single_small"])
    return cp.Planner(crane, scene, cp.make_params(N, K, S, seed=seed, sampler=sampler), stream=stream)


@pytest.mark.parametrize("sampler", [0, 1])
def test_metrics_rows_match_planner_state(lib, sampler):
    import torch
    cp = lib
    q0, qd = endpoints("single_small")
    st = torch.cuda.Stream()
    with _planner(cp, sampler, stream=st) as pl:
        h = pl.handle
        cp.cp_set_metrics(h, True)
        cp.cp_set_endpoints(h, q0, qd)
        T = 7
        _, stats = cp.cp_plan(h, T, K=pl.K)
        rows = cp.cp_get_metrics(h)
        assert rows.shape == (T, 5)
        np.testing.assert_array_equal(rows[:, 0], np.arange(T))
        last = rows[-1]
        N, K, D = pl.N, pl.K, pl.D
        with torch.cuda.stream(st):
            xi = torch.zeros(N, K, 4, device="cuda")
            J = torch.zeros(N, dtype=torch.float64, device="cuda")
            cp.cp_get_population(h, xi, J)
            J2 = torch.zeros(N, dtype=torch.float64, device="cuda")
            flag = torch.zeros(N, dtype=torch.uint8, device="cuda")
            cp.cp_evaluate(h, xi, N, J2, flag)
            C = torch.zeros(D, D, dtype=torch.float64, device="cuda")
            cp.cp_get_distribution(h, None, C)
        st.synchronize()
        Jn = J.cpu().numpy()
        assert last[1] == stats["best_J"] == Jn.min()
        np.testing.assert_allclose(last[2], Jn.mean(), rtol=1e-13)
        np.testing.assert_array_equal(J2.cpu().numpy(), Jn)
        assert last[4] == np.mean(flag.cpu().numpy() == 0)
        np.testing.assert_allclose(last[3], np.trace(C.cpu().numpy()), rtol=1e-12)
        assert np.all(rows[:, 3] > 0) and np.all((rows[:, 4] >= 0) & (rows[:, 4] <= 1))
        # the same plan kernel by kernel (timing on: no graph) gives the same rows
        cp.cp_set_timing(h, True)
        cp.cp_set_endpoints(h, q0, qd)
        cp.cp_plan(h, T, K=pl.K)
        np.testing.assert_array_equal(cp.cp_get_metrics(h), rows)
        cp.cp_set_timing(h, False)
        # off: nothing new is recorded; a new plan restarts the record
        cp.cp_set_metrics(h, False)
        cp.cp_set_endpoints(h, q0, qd)
        cp.cp_plan(h, 3)
        assert cp.cp_get_metrics(h).shape == (0, 5)


def test_metrics_ring_keeps_last_iterations(lib):
    import torch
    cp = lib
    q0, qd = endpoints("single_small")
    st = torch.cuda.Stream()
    with _planner(cp, 0, stream=st, N=64, K=2, S=4) as pl:
        h = pl.handle
        cp.cp_set_metrics(h, True)
        cp.cp_set_endpoints(h, q0, qd)
        cp.cp_plan(h, 200)
        cp.cp_plan(h, 100)          # continues from iteration 200
        rows = cp.cp_get_metrics(h, 1000)
        assert rows.shape == (256, 5)
        np.testing.assert_array_equal(rows[:, 0], np.arange(300 - 256, 300))
        assert cp.cp_get_metrics(h, 10).shape == (10, 5)
        np.testing.assert_array_equal(cp.cp_get_metrics(h, 10)[:, 0], np.arange(290, 300))


INJECTION = textwrap.dedent(r"""
    #include <stdint.h>
    #include <stdio.h>
    #include <stdlib.h>
    typedef void (*fn_t)(void);
    typedef fn_t **table_t;
    typedef struct { size_t struct_size; int (*GetModuleFunctionTable)(int, table_t *, unsigned *); } callbacks_t;
    typedef const void *(*get_export_t)(uint32_t);
    static FILE *out;
    static int push_a(const char *msg) { fprintf(out, "push %s\n", msg); fflush(out); return 0; }
    static int pop(void) { fprintf(out, "pop\n"); fflush(out); return 0; }
    int InitializeInjectionNvtx2(get_export_t get)
    {
        const callbacks_t *cb = (const callbacks_t *)get(1);      /* the callbacks table */
        table_t t = 0;
        unsigned n = 0;
        if (!cb || !cb->GetModuleFunctionTable(1, &t, &n) || n < 12) return 0;   /* core module */
        *t[9] = (fn_t)push_a;    /* RangePushA */
        *t[11] = (fn_t)pop;      /* RangePop */
        out = fopen(getenv("CP_NVTX_LOG"), "w");
        return out != 0;
    }
""")

CHILD = textwrap.dedent(r"""
    import sys
    sys.path.insert(0, {root!r})
    sys.path.insert(0, {tests!r})
    import torch
    from helpers import endpoints
    from paper_2503_14160_gb300 import craneplan as cp, workloads
    cp.load()
    crane = workloads.forestry_crane()
    scene = workloads.make_scene(workloads.WORKLOADS["single_small"])
    q0, qd = endpoints("single_small")
    with cp.Planner(crane, scene, cp.make_params(64, 4, 8)) as pl:
        cp.cp_set_timing(pl.handle, True)       # kernel by kernel: every stage enqueued each iteration
        cp.cp_set_endpoints(pl.handle, q0, qd)
        cp.cp_plan(pl.handle, 2)
    torch.cuda.synchronize()
""")


def test_nvtx_ranges_of_a_plan(lib, tmp_path):
    src = tmp_path / "inject.c"
    src.write_text(INJECTION)
    so = tmp_path / "libinject.so"
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", str(src), "-o", str(so)], check=True)
    log = tmp_path / "nvtx.log"
    child = tmp_path / "child.py"
    child.write_text(CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests")))
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(so), CP_NVTX_LOG=str(log))
    subprocess.run([sys.executable, str(child)], check=True, env=env, timeout=600)
    events = log.read_text().split("\n")
    stack, seen = [], []
    for e in events:
        if e.startswith("push "):
            stack.append(e[5:])
            seen.append("/".join(stack))
        elif e == "pop":
            assert stack, "a pop without a push"
            stack.pop()
    assert not stack, "unbalanced ranges: %s" % stack
    for path in ["craneplan:factor", "craneplan:plan/craneplan:sample", "craneplan:plan/craneplan:evaluate",
                 "craneplan:plan/craneplan:update", "craneplan:plan/craneplan:update/craneplan:factor"]:
        assert path in seen, (path, sorted(set(seen)))
    assert seen.count("craneplan:plan/craneplan:sample") == 2

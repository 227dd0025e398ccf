"""Write tests/golden/endpoints.json: the start and goal configuration of every workload,
chosen by the rule "uniform within the joint limits, rejected if in collision" with the
FP64 oracle's signed distance (clearance 1e-3 m), and the oracle's d(q) at both.

Calls only the oracle and the seeded input generator. Run from the repository root:
    python tests/golden/make_endpoints.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "oracle"))

import oracle  # noqa: E402
from paper_2503_14160_gb300 import workloads  # noqa: E402


def main():
    crane = workloads.forestry_crane()
    out = {"about": "start/goal per workload; rule: first two uniform draws within the joint "
                    "limits with oracle d(q) > 1e-3 m (seed 0, endpoint stream); "
                    "written by tests/golden/make_endpoints.py",
           "workloads": {}}
    for name, wl in workloads.WORKLOADS.items():
        scene = workloads.make_scene(wl)
        pb = oracle.Problem(crane, scene, oracle.CostParams(K=wl.n_waypoints, S=wl.substeps))
        q0, qd, ok, draws = workloads.select_endpoints(
            crane, lambda q: oracle.signed_distance(pb, q), seed=wl.seed)
        d = oracle.signed_distance(pb, [q0, qd])
        out["workloads"][name] = {"q0": [float(x) for x in q0], "qd": [float(x) for x in qd],
                                  "ok": bool(ok), "draws": int(draws),
                                  "d_q0": float(d[0]), "d_qd": float(d[1])}
        print(name, out["workloads"][name])
    with open(os.path.join(HERE, "endpoints.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

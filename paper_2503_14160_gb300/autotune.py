"""Launch-shape autotuner for the evaluation kernel.

For a problem size it times cp_evaluate under each candidate configuration (the broad-phase
form with as many CTAs per SM as fit or with 2; the exhaustive form; the uniform grid with
0.5 m or 1.0 m cells) on a synthetic population and keeps the fastest. Results are cached in a JSON file keyed by device name,
K, S and power-of-two buckets of the candidate and cylinder counts, so a batch of uneven
queries tunes each bucket once.
"""
import json
import math
import os
from typing import Dict, Optional

import numpy as np

from . import craneplan as cp
from . import workloads

CONFIGS = [
    {"grid_cell": 0.0, "eval_ctas_per_sm": 0},
    {"grid_cell": 0.0, "eval_ctas_per_sm": 2},
    {"grid_cell": 0.0, "eval_ctas_per_sm": 0, "eval_exhaustive": 1},
    {"grid_cell": 0.5, "eval_ctas_per_sm": 0},
    {"grid_cell": 1.0, "eval_ctas_per_sm": 0},
]

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "eval.json")


def _bucket(x: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, x)))))


def key(device: str, N: int, K: int, S: int, M: int) -> str:
    return "%s|K%d|S%d|N%d|M%d" % (device, K, S, _bucket(N), _bucket(M))


class Autotuner:
    def __init__(self, cache_path: Optional[str] = DEFAULT_CACHE, reps: int = 3):
        self.cache_path = cache_path
        self.reps = reps
        self.cache: Dict[str, dict] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def save(self):
        if self.cache_path:
            os.makedirs(os.path.dirname(self.cache_path), exist_ok=True)
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1)

    def best(self, crane, N: int, K: int, S: int, M: int) -> dict:
        """The fastest configuration for this size bucket (tuned on first request)."""
        import torch
        dev = torch.cuda.get_device_name()
        k = key(dev, N, K, S, M)
        if k in self.cache:
            return self.cache[k]["config"]
        Nb, Mb = min(_bucket(N), 16384), _bucket(M)
        bq = workloads.BatchQuery(Nb, K, Mb, math.sqrt(4.0 + Mb / (1.66 * math.pi)))
        scene = workloads.batch_scene(bq, seed=12345, q=0)
        q0 = np.array([0.3, 0.4, -1.2, 0.5])
        qd = np.array([-2.0, 0.6, -1.8, 1.5])
        xi = torch.from_numpy(workloads.random_candidates(q0, qd, K, Nb, seed=1)).cuda()
        J = torch.zeros(Nb, dtype=torch.float64, device="cuda")
        times = []
        for cfg in CONFIGS:
            params = cp.make_params(Nb, K, S, **cfg)
            with cp.Planner(crane, scene, params) as pl:
                cp.cp_set_endpoints(pl.handle, q0, qd)
                cp.cp_evaluate(pl.handle, xi, Nb, J)          # warm-up
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record()
                for _ in range(self.reps):
                    cp.cp_evaluate(pl.handle, xi, Nb, J)
                b.record()
                b.synchronize()
                times.append(a.elapsed_time(b) / self.reps)
        i = int(np.argmin(times))
        self.cache[k] = {"config": CONFIGS[i], "ms": times, "configs": CONFIGS}
        self.save()
        return CONFIGS[i]

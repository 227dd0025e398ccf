"""Launch-shape autotuner.

Single queries: for a problem size it times cp_evaluate under each candidate configuration
(the broad-phase form with as many CTAs per SM as fit or with 2; the exhaustive form; the
polar obstacle index with rings of 0.5 m or 1.0 m) on a synthetic population and keeps the
fastest. `best_polar` restricts the search to the polar index and its ring width (the
obstacle tile: how many listed obstacles a checkpoint's ring range takes in), the form the
batched kernels use.

Batches: `tune_batch` times the persistent batched evaluation (cp_batch_evaluate) over
block and tile shapes: CTA size (warps, i.e. candidates in flight per CTA), resident CTAs
per SM, and work items per warp in a tile (the unit a CTA takes from the device queue; an
item is G units of 32 checkpoints of one candidate, G fixed by the query). Lanes per
candidate (32) and checkpoints per lane (one per unit) are fixed by the kernels' design:
one warp owns a unit so that its sums and collision ballot are warp-wide operations.

Results are cached in a JSON file keyed by device name and size buckets, so a batch of
uneven queries tunes each bucket once. Results do not depend on any tuned value.
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

POLAR_CONFIGS = [{"grid_cell": c, "eval_ctas_per_sm": 0} for c in (0.35, 0.5, 0.75, 1.0, 1.5)]

BATCH_SHAPES = [(t, c, i) for t in (128, 256, 512) for c in (0, 1, 2) for i in (1, 2, 4, 8, 16)
                if not (t == 512 and c == 2)]

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "eval.json")


def _bucket(x: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, x)))))


def key(device: str, N: int, K: int, S: int, M: int, form: str = "") -> str:
    return "%s|K%d|S%d|N%d|M%d%s" % (device, K, S, _bucket(N), _bucket(M), form)


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

    def _tune(self, k, configs, crane, N, K, S, M) -> dict:
        import torch
        Nb, Mb = min(_bucket(N), 16384), _bucket(M)
        bq = workloads.BatchQuery(Nb, K, Mb, math.sqrt(4.0 + Mb / (1.66 * math.pi)))
        scene = workloads.batch_scene(bq, seed=12345, q=0)
        q0 = np.array([0.3, 0.4, -1.2, 0.5])
        qd = np.array([-2.0, 0.6, -1.8, 1.5])
        xi = torch.from_numpy(workloads.random_candidates(q0, qd, K, Nb, seed=1)).cuda()
        J = torch.zeros(Nb, dtype=torch.float64, device="cuda")
        times = []
        for cfg in configs:
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
        self.cache[k] = {"config": configs[i], "ms": times, "configs": configs}
        self.save()
        return configs[i]

    def best(self, crane, N: int, K: int, S: int, M: int) -> dict:
        """The fastest configuration for this size bucket (tuned on first request)."""
        import torch
        k = key(torch.cuda.get_device_name(), N, K, S, M)
        if k in self.cache:
            return self.cache[k]["config"]
        return self._tune(k, CONFIGS, crane, N, K, S, M)

    def best_polar(self, crane, N: int, K: int, S: int, M: int) -> dict:
        """The fastest ring width of the polar index for this size bucket."""
        import torch
        k = key(torch.cuda.get_device_name(), N, K, S, M, "|polar")
        if k in self.cache:
            return self.cache[k]["config"]
        return self._tune(k, POLAR_CONFIGS, crane, N, K, S, M)

    def tune_batch(self, b: int, signature: str, reps: int = 3) -> dict:
        """Time the batch's persistent evaluation under every shape of BATCH_SHAPES (the
        populations the batch holds, e.g. after a run), set the fastest on the batch and
        cache it under `signature` (a description of the batch's sizes)."""
        import torch
        k = "%s|batch|%s" % (torch.cuda.get_device_name(), signature)
        if k in self.cache:
            best = self.cache[k]["shape"]
            cp.cp_batch_set_shape(b, *best)
            return self.cache[k]
        times = []
        for shape in BATCH_SHAPES:
            cp.cp_batch_set_shape(b, *shape)
            cp.cp_batch_evaluate(b, 1)                       # warm-up
            times.append(cp.cp_batch_evaluate(b, reps))
        i = int(np.argmin(times))
        cp.cp_batch_set_shape(b, *BATCH_SHAPES[i])
        self.cache[k] = {"shape": list(BATCH_SHAPES[i]), "ms": times,
                         "shapes": [list(s) for s in BATCH_SHAPES]}
        self.save()
        return self.cache[k]

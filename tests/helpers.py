"""Shared set-up for the GPU parity tests: planners, oracle problems and tolerances.

Tolerances (FP32 kernels against the FP64 oracle on identical inputs):
  D_TOL      bound on |d_gpu - d_oracle| per checkpoint (m). Sphere centres come from FP32
             kinematics over lever arms up to ~10 m (a few ulp of 10 m, ~1e-6 m each);
             the distance itself is a few more FP32 operations. 2e-5 m leaves margin and
             stays well below the 1e-4 m band outside which flags must agree bit for bit.
  FLAG_BAND  |d| above which per-checkpoint collision flags must agree exactly (1e-4 m).
  J_REL      relative tolerance on J for the smooth parts (1e-4); the collision term adds
             an absolute allowance lambda_c * w_c * D_TOL per checkpoint whose oracle
             distance is below D_TOL (penetrating or grazing), because max(0, -d) there
             carries the distance error unchanged.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "oracle"))

D_TOL = 2e-5
FLAG_BAND = 1e-4
J_REL = 1e-4


def endpoints(name):
    with open(os.path.join(ROOT, "tests", "golden", "endpoints.json")) as f:
        e = json.load(f)["workloads"][name]
    return np.array(e["q0"]), np.array(e["qd"])


def cost_tolerance(J_oracle, n_near, w_c=100.0, lambda_c=1.0):
    return J_REL * np.abs(J_oracle) + w_c * lambda_c * D_TOL * n_near + 1e-9


def unpack_flags(words, n_s):
    """uint32[n][W] -> bool[n][n_s] (bit b of word w is checkpoint 32 w + b + 1)."""
    w = np.asarray(words, dtype=np.uint32)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)[None, None, :]) & 1).astype(bool)
    return bits.reshape(w.shape[0], -1)[:, :n_s]


class Setup:
    """A GPU planner and the matching oracle problem for one scene and size."""

    def __init__(self, crane, scene, N, K, S, seed=0, n_elites=0, w_c=100.0, w_l=100.0,
                 lambda_c=1.0, eps=1e-8, sigma=1.0, grid_cell=0.0, grid_half_extent=0.0,
                 exhaustive=0, update_rule=0, sampler=0):
        import torch
        import oracle
        from paper_2503_14160_gb300 import craneplan as cp
        self.torch, self.cp, self.oracle = torch, cp, oracle
        self.crane, self.scene = crane, scene
        self.N, self.K, self.S = N, K, S
        self.n_s = (K + 3) * S
        self.D = 4 * K
        params = cp.make_params(N, K, S, n_elites=n_elites, w_c=w_c, w_l=w_l,
                                lambda_c=lambda_c, eps=eps, sigma=sigma, seed=seed,
                                grid_cell=grid_cell, grid_half_extent=grid_half_extent,
                                eval_exhaustive=exhaustive, update_rule=update_rule, sampler=sampler)
        self.planner = cp.Planner(crane, scene, params)
        self.nu = self.planner.nu
        self.problem = oracle.Problem(crane, scene, oracle.CostParams(K=K, S=S, w_c=w_c, w_l=w_l,
                                                                      lambda_c=lambda_c))
        self.sp = oracle.SearchParams(N=N, K=K, S=S, nu=n_elites, sigma=sigma, eps=eps, seed=seed)

    @property
    def h(self):
        return self.planner.handle

    def evaluate(self, xi_np, q0, qd):
        """GPU evaluation of float32 candidates; returns dict of numpy arrays."""
        torch, cp = self.torch, self.cp
        cp.cp_set_endpoints(self.h, q0, qd)
        n = xi_np.shape[0]
        xi = torch.from_numpy(np.ascontiguousarray(xi_np, np.float32)).cuda()
        J = torch.zeros(n, dtype=torch.float64, device="cuda")
        flag = torch.zeros(n, dtype=torch.uint8, device="cuda")
        terms = torch.zeros(n, 5, dtype=torch.float64, device="cuda")
        W = (self.n_s + 31) // 32
        words = torch.zeros(n, W, dtype=torch.int32, device="cuda")
        pen = torch.zeros(n, self.n_s, dtype=torch.float32, device="cuda")
        cp.cp_evaluate(self.h, xi, n, J, flag, terms, words, pen)
        torch.cuda.synchronize()
        return {"J": J.cpu().numpy(), "flag": flag.cpu().numpy(), "terms": terms.cpu().numpy(),
                "words": words.cpu().numpy().view(np.uint32), "pen": pen.cpu().numpy()}

    def close(self):
        self.planner.close()


EPS32 = 2.0 ** -24


def factor_sample_bound(want, z, L):
    """Float32 bound of a draw mu + L z against its FP64 value: the result's rounding and a
    D-term float32 dot product of L and z."""
    D = L.shape[0]
    return EPS32 * np.abs(want) + (D + 8) * EPS32 * (np.abs(z[:, :D]) @ np.abs(L).T) + 1e-30


def elite_sample_bound(want, z, X, mu, w, sigma, eps, slices=32):
    """Worst-case bound of the tensor-core elite draw (3xTF32 products accumulated in FP32)
    against the oracle's FP64 sample_elites, per coordinate; also returns the scale
    sum_j |g_ij||Y_jd| used by the RMS check (see test_gpu_sample_elites)."""
    nu, D = X.shape
    Y = np.sqrt(w)[:, None] * (X - mu[None, :]) * sigma
    scale = np.abs(z[:, :nu]) @ np.abs(Y)
    bound = (EPS32 * np.abs(want) + (20 + 6 * nu + slices + 16) * EPS32 * scale
             + 8 * EPS32 * sigma * np.sqrt(eps) * np.abs(z[:, nu:nu + D]) + 1e-30)
    return bound, scale

"""torch.autograd.Function around the smooth path cost and its hand-written adjoint kernel.

PathCost.apply(xi, planner) returns J_s for candidates xi (float32 CUDA tensor [n][K][4]);
backward calls cp_smooth_cost_grad, which returns dJ_s/dxi scaled by the incoming gradient.
Both directions run in the CUDA library; this file only marshals tensors.
"""
import torch

from . import craneplan as cp


class PathCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xi: torch.Tensor, planner) -> torch.Tensor:
        xi = xi.contiguous()
        if xi.dtype != torch.float32 or not xi.is_cuda:
            raise TypeError("xi must be a float32 CUDA tensor [n][K][4]")
        n = xi.shape[0]
        J = torch.empty(n, dtype=torch.float64, device=xi.device)
        cp.cp_smooth_cost(planner.handle, xi, n, J)
        ctx.save_for_backward(xi)
        ctx.planner = planner
        return J

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        (xi,) = ctx.saved_tensors
        dxi = torch.empty_like(xi)
        gJ = gJ.detach().to(torch.float64).contiguous()
        cp.cp_smooth_cost_grad(ctx.planner.handle, xi, xi.shape[0], gJ, None, dxi)
        return dxi, None


def path_cost(xi: torch.Tensor, planner) -> torch.Tensor:
    return PathCost.apply(xi, planner)

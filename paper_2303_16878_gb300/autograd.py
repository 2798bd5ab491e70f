"""Differentiable total photometric cost (Eq. total-error-multicue) for PyTorch.

`photometric_cost(problem, poses, extrinsics, channels)` returns F as a
0-dim float64 CUDA tensor.  Its backward launches the library's adjoint
kernel (pba_cost_gradient), which recomputes every projection and sample
instead of keeping per-residual Jacobians, and returns dF/dposes (N, 3, 4),
dF/dX_o (S, 3, 4) and dF/dchannels (N, H, W, 5).  The pair list, intrinsics,
weights and thresholds are the problem's; the validity decisions are held
fixed (F is piecewise smooth).  All frames must share one image size.
"""
from __future__ import annotations

import torch


def _apply(problem, poses, extrinsics, channels):
    problem.set_poses(poses.detach().contiguous())
    for s in range(extrinsics.shape[0]):
        problem.set_extrinsic(s, extrinsics[s])
    problem.upload_frames(0, channels.detach().contiguous())


class PhotometricCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, poses, extrinsics, channels, problem):
        _apply(problem, poses, extrinsics, channels)
        cost, _, _, _, _ = problem.cost_gradient(poses=False, extrinsics=False, images=False, device=poses.device)
        ctx.problem = problem
        ctx.save_for_backward(poses, extrinsics, channels)
        return torch.tensor(cost, dtype=torch.float64, device=poses.device)

    @staticmethod
    def backward(ctx, grad):
        poses, extrinsics, channels = ctx.saved_tensors
        problem = ctx.problem
        _apply(problem, poses, extrinsics, channels)  # the problem may have moved since the forward
        need_p, need_e, need_i = ctx.needs_input_grad[:3]
        _, _, dP, dE, dI = problem.cost_gradient(poses=need_p, extrinsics=need_e, images=need_i,
                                                 device=poses.device)
        g = grad.to(torch.float64)
        out_p = (g * dP).to(poses.dtype) if need_p else None
        out_e = (g * dE).to(extrinsics.dtype) if need_e else None
        out_i = (g.to(torch.float32) * dI).view_as(channels) if need_i else None
        return out_p, out_e, out_i, None


def photometric_cost(problem, poses, extrinsics, channels):
    """F(poses, extrinsics, channels) with the adjoint as its backward."""
    return PhotometricCost.apply(poses, extrinsics, channels, problem)


def tangent_gradient(problem, poses, dposes):
    """dF/d dx_k in the box-plus chart of the Supp. from the matrix gradient
    dF/dX_k at the poses X_k: the library's pba_tangent_gradient on the
    device ((N, 3, 4), (N, 3, 4) -> (N, 6))."""
    return problem.tangent_gradient(poses, dposes)

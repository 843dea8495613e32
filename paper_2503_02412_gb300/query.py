"""Continuous SE(2) pose query with a hand-written backward kernel, as a torch.autograd.Function.

forward: poses [N, 3] (x, y, yaw; world metres / rad) -> out [N, 5] (z, pitch, roll, rough,
risk) and flags [N] (uint8), via seb_query_poses.  backward: seb_query_poses_backward, the
adjoint kernel, with the valid footprint points held fixed and zero gradient on the clamped
risk = 1 branches.  Both kernels run in libseb; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import abi
from .maps import SebParams


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def query_poses(params: SebParams, elev: torch.Tensor, poses: torch.Tensor, origin=(0, 0), saved=None):
    """Forward only.  Returns (out [N, 5] float32, flags [N] uint8)."""
    _check(params, elev, poses)
    n = poses.shape[0]
    out = torch.empty((n, 5), dtype=torch.float32, device=poses.device)
    flags = torch.empty((n,), dtype=torch.uint8, device=poses.device)
    abi.seb_query_poses(params.c(), elev.data_ptr(), int(origin[0]), int(origin[1]), poses.data_ptr(), n,
                        out.data_ptr(), flags.data_ptr(), saved.data_ptr() if saved is not None else 0,
                        _stream(poses))
    return out, flags


def _check(params, elev, poses):
    if not (elev.is_cuda and poses.is_cuda):
        raise ValueError("elevation and poses must be CUDA tensors")
    if elev.dtype != params.elev_dtype or tuple(elev.shape) != (params.ny, params.nx) or not elev.is_contiguous():
        raise ValueError(f"elevation must be a contiguous {params.elev_dtype} tensor of shape ({params.ny}, {params.nx})")
    if poses.dtype != torch.float32 or poses.dim() != 2 or poses.shape[1] != 3 or not poses.is_contiguous():
        raise ValueError("poses must be a contiguous float32 tensor [N, 3]")


class QueryPoses(torch.autograd.Function):
    """out, flags = QueryPoses.apply(poses, elev, params, origin)."""

    @staticmethod
    def forward(ctx, poses, elev, params, origin=(0, 0)):
        poses = poses.contiguous()
        saved = torch.empty((poses.shape[0], abi.SEB_QUERY_SAVED), dtype=torch.float32, device=poses.device)
        out, flags = query_poses(params, elev, poses, origin, saved)
        ctx.save_for_backward(poses, elev, saved)
        ctx.params = params
        ctx.origin = origin
        ctx.mark_non_differentiable(flags)
        return out, flags

    @staticmethod
    def backward(ctx, grad_out, _grad_flags):
        poses, elev, saved = ctx.saved_tensors
        p = ctx.params
        g = grad_out.contiguous().to(torch.float32)
        gp = torch.empty_like(poses)
        abi.seb_query_poses_backward(p.c(), elev.data_ptr(), int(ctx.origin[0]), int(ctx.origin[1]),
                                     poses.data_ptr(), saved.data_ptr(), g.data_ptr(), gp.data_ptr(),
                                     poses.shape[0], _stream(poses))
        return gp, None, None, None

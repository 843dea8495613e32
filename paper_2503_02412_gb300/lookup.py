"""Trilinear SE(2) grid lookup with gradients, as used by the paper's planner (Sec. VI: Risk and
the signed distance field are read at continuous states by trilinear interpolation, with the yaw
on SO(2)).

``SE2Grid`` names one ring-indexed [n_yaw][ny][nx] float32 channel on the device: a channel of
a ``SebMap`` (``SE2Grid.from_map``) or any caller tensor (``SE2Grid.from_tensor``).
``se2_lookup`` returns values, optional world-unit gradients and flags; ``SE2Lookup`` is the
differentiable form whose backward runs the adjoint kernel; ``risk_sdf`` builds the signed
distance field of the obstacle set as another grid.  The kernels are libseb's
(``seb_se2_lookup``, ``seb_se2_lookup_vjp``, ``seb_risk_sdf``); this module only marshals
tensors.
"""
from __future__ import annotations

import math

import torch

from . import abi


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


class SE2Grid:
    """A seb_grid plus a reference to the storage that backs it."""

    def __init__(self, g: "abi.seb_grid", owner, device):
        self.g = g
        self._owner = owner  # keeps the map or tensor alive
        self.device = device

    @classmethod
    def from_map(cls, m, channel: int) -> "SE2Grid":
        """Channel 0..4 (z, pitch, roll, roughness, risk) of a map's current outputs; valid until
        its next update or shift."""
        return cls(abi.seb_map_grid(m.handle, int(channel)), m, m.device)

    @classmethod
    def from_tensor(cls, data: torch.Tensor, res: float, origin=(0, 0), ring=(0, 0)) -> "SE2Grid":
        if not data.is_cuda or data.dtype != torch.float32 or data.dim() != 3 or not data.is_contiguous():
            raise ValueError("grid must be a contiguous float32 CUDA tensor [n_yaw, ny, nx]")
        K, ny, nx = data.shape
        g = abi.seb_grid(data.data_ptr(), nx, ny, K, int(ring[0]), int(ring[1]), int(origin[0]), int(origin[1]),
                         float(res))
        return cls(g, data, data.device)


def _check_poses(poses: torch.Tensor):
    if not poses.is_cuda or poses.dtype != torch.float32 or poses.dim() != 2 or poses.shape[1] != 3:
        raise ValueError("poses must be a float32 CUDA tensor [N, 3]")


def se2_lookup(grid: SE2Grid, poses: torch.Tensor, fill: float = math.nan, with_grad: bool = False):
    """Returns (value [N], grad [N, 3] or None, flags [N] uint8)."""
    _check_poses(poses)
    poses = poses.contiguous()
    n = poses.shape[0]
    val = torch.empty((n,), dtype=torch.float32, device=poses.device)
    grad = torch.empty((n, 3), dtype=torch.float32, device=poses.device) if with_grad else None
    flags = torch.empty((n,), dtype=torch.uint8, device=poses.device)
    abi.seb_se2_lookup(grid.g, poses.data_ptr(), n, float(fill), val.data_ptr(),
                       grad.data_ptr() if grad is not None else None, flags.data_ptr(), _stream(poses))
    return val, grad, flags


def risk_sdf(risk: SE2Grid, risk_obstacle: float = 1.0, clamp: float = math.inf, out: torch.Tensor = None,
             work: torch.Tensor = None) -> SE2Grid:
    """Signed distance field (metres) of the obstacle set (risk >= risk_obstacle) of every yaw
    bin of a risk grid, stored ring-indexed like it; returns it as an SE2Grid for lookups."""
    g = risk.g
    shape = (g.n_yaw, g.ny, g.nx)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=risk.device)
    if tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous float32 tensor of shape {shape}")
    nb = abi.seb_sdf_workspace_bytes(g.nx, g.ny, g.n_yaw)
    if work is None or work.numel() * work.element_size() < nb:
        work = torch.empty(nb, dtype=torch.uint8, device=risk.device)
    abi.seb_risk_sdf(g, float(risk_obstacle), float(clamp), work.data_ptr(), nb, out.data_ptr(),
                     _stream(out))
    sg = abi.seb_grid(out.data_ptr(), g.nx, g.ny, g.n_yaw, g.ring_x, g.ring_y, g.origin_i, g.origin_j, g.res)
    return SE2Grid(sg, out, risk.device)


class SE2Lookup(torch.autograd.Function):
    """value = SE2Lookup.apply(poses, grid, fill): differentiable in the poses."""

    @staticmethod
    def forward(ctx, poses, grid, fill=math.nan):
        poses = poses.contiguous()
        val, _, _ = se2_lookup(grid, poses, fill)
        ctx.save_for_backward(poses)
        ctx.grid = grid
        return val

    @staticmethod
    def backward(ctx, grad_val):
        (poses,) = ctx.saved_tensors
        g = grad_val.contiguous().to(torch.float32)
        gp = torch.empty_like(poses)
        abi.seb_se2_lookup_vjp(ctx.grid.g, poses.data_ptr(), poses.shape[0], g.data_ptr(), gp.data_ptr(),
                               _stream(poses))
        return gp, None, None

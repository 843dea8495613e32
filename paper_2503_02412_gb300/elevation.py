"""Elevation-map update from LiDAR scans (Sec. V-A): robot-centred window, ray-casting clearing,
point filtering, per-point height variance and one-dimensional Kalman fusion, all in libseb's
``seb_elev_*`` kernels; this module only marshals tensors and the pose."""
from __future__ import annotations

import numpy as np
import torch

from . import abi


def _f9(m):
    return (abi.ctypes.c_float * 9)(*np.asarray(m, np.float64).reshape(9).tolist())


def _f3(v):
    return (abi.ctypes.c_float * 3)(*np.asarray(v, np.float64).reshape(3).tolist())


def scan_pose(R_B, p_B, R_BS, p_BS, Sigma_S, Sigma_R, Sigma_B) -> "abi.seb_scan_pose":
    return abi.seb_scan_pose(_f9(R_B), _f3(p_B), _f9(R_BS), _f3(p_BS), _f9(Sigma_S), _f9(Sigma_R), _f9(Sigma_B))


class ElevationMap:
    def __init__(self, nx, ny, res, max_points, z_min=-1.0, z_max=1.0, gate=2.5, clear_margin=0.05, device="cuda"):
        self.device = torch.device(device)
        self.p = abi.seb_elev_params(nx, ny, res, z_min, z_max, gate, clear_margin)
        nb = abi.seb_elev_workspace_bytes(self.p, max_points)
        if nb == 0:
            raise ValueError("invalid elevation-map parameters")
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.handle = abi.seb_elev_create(self.p, max_points, self.workspace.data_ptr(), nb, self._stream())
        self.max_points = max_points

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            abi.seb_elev_destroy(h)
            self.handle = None

    def integrate(self, pose: "abi.seb_scan_pose", points: torch.Tensor):
        if not points.is_cuda or points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 3:
            raise ValueError("points must be a float32 CUDA tensor [n, 3]")
        points = points.contiguous()
        abi.seb_elev_set_stream(self.handle, self._stream())
        abi.seb_elev_integrate(self.handle, pose, points.data_ptr(), points.shape[0])

    def view(self):
        return abi.seb_elev_view_get(self.handle)

    def outputs(self, height: torch.Tensor = None, variance: torch.Tensor = None):
        """(height, variance) [ny, nx] in window order."""
        shape = (self.p.ny, self.p.nx)
        if height is None:
            height = torch.empty(shape, dtype=torch.float32, device=self.device)
        if variance is None:
            variance = torch.empty(shape, dtype=torch.float32, device=self.device)
        abi.seb_elev_set_stream(self.handle, self._stream())
        abi.seb_elev_copy_out(self.handle, height.data_ptr(), variance.data_ptr())
        return height, variance

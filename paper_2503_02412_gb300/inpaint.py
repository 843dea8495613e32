"""Nearest-neighbour inpainting of an elevation map before the traversability pass (Sec. V-A;
Sec. VII-B uses nearest-neighbour filling).  The kernels are libseb's (``seb_inpaint_nearest``);
this module only marshals tensors."""
from __future__ import annotations

import torch

from . import abi


def inpaint_nearest(elev: torch.Tensor, max_cells: int = 0, out: torch.Tensor = None, work: torch.Tensor = None,
                    with_source: bool = False):
    """elev [ny, nx] float32 CUDA (NaN = unknown) -> filled [ny, nx] (and the source (row, col)
    of every value, [ny, nx, 2] int32, when with_source)."""
    if not elev.is_cuda or elev.dtype != torch.float32 or elev.dim() != 2 or not elev.is_contiguous():
        raise ValueError("elevation must be a contiguous float32 CUDA tensor [ny, nx]")
    ny, nx = elev.shape
    if out is None:
        out = torch.empty_like(elev)
    nb = abi.seb_inpaint_workspace_bytes(nx, ny)
    if work is None or work.numel() * work.element_size() < nb:
        work = torch.empty(nb, dtype=torch.uint8, device=elev.device)
    src = torch.empty((ny, nx, 2), dtype=torch.int32, device=elev.device) if with_source else None
    abi.seb_inpaint_nearest(elev.data_ptr(), nx, ny, int(max_cells), work.data_ptr(), nb, out.data_ptr(),
                            src.data_ptr() if src is not None else None,
                            torch.cuda.current_stream(elev.device).cuda_stream)
    return (out, src) if with_source else out

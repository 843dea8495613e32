"""PyTorch-facing wrapper of a libseb map: torch owns the device workspace and supplies the
stream; libseb's kernels do all the work (SEB-Naver Sec. V, Algorithm 1)."""
from __future__ import annotations

import dataclasses

import torch

from . import abi

DTYPES = {torch.float32: abi.SEB_F32, torch.bfloat16: abi.SEB_BF16, torch.float16: abi.SEB_F16,
          "bf16_tiled": abi.SEB_BF16_TILED}
TILE = 16  # SEB_BF16_TILED: world-aligned tiles of 16 x 16 cells
CHANNELS = ("z", "pitch", "roll", "rough", "risk")


@dataclasses.dataclass
class SebParams:
    """Mirror of the C ``seb_params``.  phi limits default to 0.52 rad (Sec. VII-B);
    kappa_max, the weights and the footprint extents are the caller's choice."""

    nx: int = 100
    ny: int = 100
    n_yaw: int = 36
    res: float = 0.1
    length: float = 0.6
    width: float = 0.4
    shape: str = "rect"
    kappa_max: float = 0.1
    phi_x_max: float = 0.52
    phi_y_max: float = 0.52
    w: tuple = (1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)
    n_min: int = 0
    elev_dtype: torch.dtype = torch.float32
    precision: str = "plain"  # "plain" | "compensated"
    gap_fp64: float = 1e-2

    def c(self) -> abi.seb_params:
        p = abi.seb_params()
        p.nx, p.ny, p.n_yaw = self.nx, self.ny, self.n_yaw
        p.res = self.res
        p.shape = {"rect": abi.SEB_RECT, "ellipse": abi.SEB_ELLIPSE}[self.shape]
        p.length, p.width = self.length, self.width
        p.kappa_max, p.phi_x_max, p.phi_y_max = self.kappa_max, self.phi_x_max, self.phi_y_max
        for i in range(3):
            p.w[i] = self.w[i]
        p.n_min = self.n_min
        p.elev_dtype = DTYPES[self.elev_dtype]
        p.precision = {"plain": abi.SEB_PLAIN_F32, "compensated": abi.SEB_COMPENSATED}[self.precision]
        p.gap_fp64 = self.gap_fp64
        return p


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class SebMap:
    """A rolling SE(2) traversability map.  ``update`` rebuilds every cell, ``shift`` moves
    the window and recomputes only the affected bands; ``outputs()`` returns the logical
    [5][n_yaw][ny][nx] view (a ring-unrolled copy) and the flags."""

    def __init__(self, params: SebParams, device="cuda"):
        self.params = params
        self.device = torch.device(device)
        self._p = params.c()
        nbytes = abi.seb_workspace_bytes(self._p)
        if nbytes == 0:
            raise ValueError("invalid map parameters")
        # 256-byte alignment: torch's caching allocator returns 512-byte aligned blocks.
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.handle = abi.seb_map_create(self._p, self.workspace.data_ptr(), nbytes, _stream(self.device))
        v = abi.seb_map_view(self.handle)
        K, ny, nx = params.n_yaw, params.ny, params.nx
        n = 5 * K * ny * nx
        self.out_phys = self.workspace[v.out_offset:v.out_offset + 4 * n].view(torch.float32).view(5, K, ny, nx)
        self.flags_phys = self.workspace[v.flags_offset:v.flags_offset + K * ny * nx].view(K, ny, nx)
        self._elev = None

    def close(self):
        if getattr(self, "handle", None):
            abi.seb_map_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_elev(self, elev):
        p = self.params
        if p.elev_dtype == "bf16_tiled":
            n = abi.seb_window_bytes(self._p)
            if elev.dtype != torch.uint8 or elev.numel() != n or not elev.is_cuda or not elev.is_contiguous():
                raise ValueError(f"a bf16_tiled window is a contiguous CUDA uint8 tensor of {n} bytes "
                                 "(encode_bf16_tiled / tiled_window)")
            self._elev = elev
            return
        if elev.dtype != p.elev_dtype or tuple(elev.shape) != (p.ny, p.nx) or not elev.is_cuda:
            raise ValueError(f"elevation must be a CUDA {p.elev_dtype} tensor of shape ({p.ny}, {p.nx})")
        if not elev.is_contiguous():
            raise ValueError("elevation must be contiguous")
        self._elev = elev  # keep alive while kernels may read it

    def update(self, elev: torch.Tensor, origin=(0, 0)):
        self._check_elev(elev)
        abi.seb_map_set_stream(self.handle, _stream(self.device))
        abi.seb_map_update(self.handle, elev.data_ptr(), int(origin[0]), int(origin[1]))

    def shift(self, elev: torch.Tensor, origin):
        self._check_elev(elev)
        abi.seb_map_set_stream(self.handle, _stream(self.device))
        abi.seb_map_shift(self.handle, elev.data_ptr(), int(origin[0]), int(origin[1]))

    def shift_batch(self, elevs, origins):
        """Rolling updates to origins[i] with windows elevs[i], in order; bit-identical to
        calling shift for each.  The windows must all be written before the call and stay
        untouched until its work on the stream has completed."""
        if len(elevs) != len(origins):
            raise ValueError("one origin per window")
        for e in elevs:
            self._check_elev(e)
        abi.seb_map_set_stream(self.handle, _stream(self.device))
        abi.seb_map_shift_batch(self.handle, [e.data_ptr() for e in elevs], [(int(o[0]), int(o[1])) for o in origins])

    def view(self):
        return abi.seb_map_view(self.handle)

    def outputs(self, out: torch.Tensor = None, fl: torch.Tensor = None):
        """Logical-order copy: (out [5][K][ny][nx] float32, flags [K][ny][nx] uint8), into the
        given contiguous tensors when provided."""
        p = self.params
        if out is None:
            out = torch.empty((5, p.n_yaw, p.ny, p.nx), dtype=torch.float32, device=self.device)
        if fl is None:
            fl = torch.empty((p.n_yaw, p.ny, p.nx), dtype=torch.uint8, device=self.device)
        if tuple(out.shape) != (5, p.n_yaw, p.ny, p.nx) or not out.is_contiguous() or out.dtype != torch.float32:
            raise ValueError("out must be a contiguous float32 tensor [5, n_yaw, ny, nx]")
        if tuple(fl.shape) != (p.n_yaw, p.ny, p.nx) or not fl.is_contiguous() or fl.dtype != torch.uint8:
            raise ValueError("flags must be a contiguous uint8 tensor [n_yaw, ny, nx]")
        abi.seb_map_set_stream(self.handle, _stream(self.device))
        abi.seb_map_copy_out(self.handle, out.data_ptr(), fl.data_ptr())
        return out, fl

    def check(self, timeout_ms=10000):
        abi.seb_map_set_stream(self.handle, _stream(self.device))
        return abi.seb_map_check(self.handle, timeout_ms)


def encode_bf16_tiled(elev: torch.Tensor, origin=(0, 0)) -> torch.Tensor:
    """FP32 elevation [ny][nx] on the device -> a SEB_BF16_TILED window buffer (uint8): BF16
    offsets from an FP32 base per 16 x 16 world-aligned tile (seb_encode_bf16_tiled)."""
    if elev.dtype != torch.float32 or elev.dim() != 2 or not elev.is_cuda or not elev.is_contiguous():
        raise ValueError("elevation must be a contiguous CUDA float32 [ny][nx] tensor")
    ny, nx = elev.shape
    p = SebParams(nx=nx, ny=ny, elev_dtype="bf16_tiled").c()
    out = torch.empty(abi.seb_window_bytes(p), dtype=torch.uint8, device=elev.device)
    abi.seb_encode_bf16_tiled(elev.data_ptr(), nx, ny, int(origin[0]), int(origin[1]), out.data_ptr(),
                              _stream(elev.device))
    return out


def tiled_parts(buf: torch.Tensor, nx: int, ny: int):
    """Views of a SEB_BF16_TILED buffer: (offsets [ny][nx] bfloat16, bases [TY][TX] float32)."""
    off = abi.seb_tiled_base_offset(nx, ny)
    tx, ty = (nx + TILE - 1) // TILE + 1, (ny + TILE - 1) // TILE + 1
    return (buf[:nx * ny * 2].view(torch.bfloat16).view(ny, nx),
            buf[off:off + 4 * tx * ty].view(torch.float32).view(ty, tx))


def tiled_window(world: torch.Tensor, world_nx: int, world_ny: int, oi: int, oj: int, nx: int, ny: int) -> torch.Tensor:
    """Cuts the window at world cell (oi, oj) (0 <= oi, oi + nx <= world_nx, same for rows) of
    size nx x ny out of a SEB_BF16_TILED encoding of a whole world made at origin (0, 0)."""
    wd, wb = tiled_parts(world, world_nx, world_ny)
    p = SebParams(nx=nx, ny=ny, elev_dtype="bf16_tiled").c()
    out = torch.zeros(abi.seb_window_bytes(p), dtype=torch.uint8, device=world.device)
    d, b = tiled_parts(out, nx, ny)
    d.copy_(wd[oj:oj + ny, oi:oi + nx])
    bt = wb[oj // TILE:oj // TILE + b.shape[0], oi // TILE:oi // TILE + b.shape[1]]
    b[:bt.shape[0], :bt.shape[1]].copy_(bt)
    return out

"""Learned BF16 surrogate of the SE(2) assessment, trained on the GPU on patches the exact
kernel labels (libseb's seb_sur_* kernels), and run over a map with the exact kernel as
fallback.  This module only draws the random terrain parameters and patch centres and
marshals tensors; every numerical step runs in libseb."""
from __future__ import annotations

import math

import numpy as np
import torch

from . import abi
from .maps import SebMap, SebParams

TERRAIN_PARAMS = 36


def terrain_params(rng, n, size_m, noise=0.01):
    """Small-map recipe per world: tilt tan(U[0, 15 deg]) at a random azimuth, 8 Gaussian bumps
    (amplitude U[-0.5, 0.5] m, sigma U[0.3, 1.5] m, centres uniform) and N(0, noise) noise."""
    p = np.zeros((n, TERRAIN_PARAMS), np.float32)
    p[:, 0] = np.tan(np.deg2rad(rng.uniform(0, 15, n)))
    p[:, 1] = rng.uniform(0, 2 * math.pi, n)
    p[:, 2] = noise
    for j in range(8):
        q = 4 + 4 * j
        p[:, q] = rng.uniform(-0.5, 0.5, n)
        p[:, q + 1] = rng.uniform(0.3, 1.5, n)
        p[:, q + 2] = rng.uniform(0, size_m, n)
        p[:, q + 3] = rng.uniform(0, size_m, n)
    return p


class Surrogate:
    """params: the exact assessment to imitate and the map size used for inference."""

    def __init__(self, params: SebParams, max_batch=256, device="cuda", world=200):
        if params.elev_dtype != torch.float32:
            raise ValueError("the surrogate reads FP32 elevation")
        self.params = params
        self.device = torch.device(device)
        self.max_batch = max_batch
        self._p = params.c()
        nb = abi.seb_sur_workspace_bytes(self._p, max_batch)
        if nb == 0:
            raise ValueError("invalid surrogate parameters")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.handle = abi.seb_sur_create(self._p, max_batch, self.ws.data_ptr(), nb, self._stream())
        self.v = abi.seb_sur_view_get(self.handle)
        self.n_params = self.v.n_params
        self.n_out = self.v.n_out
        # training worlds: world x world cells at the assessment's resolution
        self.world = world
        wp = SebParams(**{**params.__dict__, "nx": world, "ny": world})
        self.label_map = SebMap(wp, self.device)
        K = params.n_yaw
        self.exact = torch.empty((5, K, world, world), dtype=torch.float32, device=self.device)
        self.exact_flags = torch.empty((K, world, world), dtype=torch.uint8, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step = 0

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def _f32(self, off, n):
        return self.ws[off:off + 4 * n].view(torch.float32)

    def _bf16(self, off, n):
        return self.ws[off:off + 2 * n].view(torch.bfloat16)

    # views into the workspace
    @property
    def master(self):
        return self._f32(self.v.master, self.n_params)

    @property
    def grad(self):
        return self._f32(self.v.grad, self.n_params)

    @property
    def weights_bf16(self):
        return self._bf16(self.v.weights_bf16, self.n_params)

    def features(self, b):
        return self._bf16(self.v.features, b * 46 * 46 * 2).view(b, 46, 46, 2)

    def labels(self, b):
        return self._f32(self.v.labels, b * 256 * self.n_out).view(b, 16, 16, self.n_out)

    def pred(self, b):
        return self._f32(self.v.pred, b * 256 * self.n_out).view(b, 16, 16, self.n_out)

    def act(self, l, b):
        side = (44, 40, 32, 16)[l]
        return self._bf16(self.v.act[l], b * side * side * 32).view(b, side, side, 32)

    def set_engine(self, engine: str):
        """"simt" or "tcgen05" for the 32 -> 32 convolutions."""
        abi.seb_sur_set_engine(self.handle, {"simt": abi.SEB_SUR_SIMT, "tcgen05": abi.SEB_SUR_TCGEN05}[engine])

    def init(self, seed=0):
        abi.seb_sur_set_stream(self.handle, self._stream())
        abi.seb_sur_init(self.handle, seed)
        self.step = 0

    def make_batch(self, rng, batch, patches_per_world=64):
        """Generates terrain on the GPU, labels it with the exact kernel and gathers `batch`
        patches (64 per world)."""
        s = self._stream()
        abi.seb_sur_set_stream(self.handle, s)
        n_worlds = (batch + patches_per_world - 1) // patches_per_world
        prm = torch.from_numpy(terrain_params(rng, n_worlds, self.world * self.params.res)).to(self.device)
        worlds = torch.empty((n_worlds, self.world, self.world), dtype=torch.float32, device=self.device)
        abi.seb_terrain_bumpy(prm.data_ptr(), n_worlds, self.world, self.world, self.params.res,
                              int(rng.integers(1 << 62)), worlds.data_ptr(), s)
        lo, hi = 24, self.world - 24
        off = 0
        for w in range(n_worlds):
            n = min(patches_per_world, batch - off)
            self.label_map.update(worlds[w], (0, 0))
            abi.seb_map_copy_out(self.label_map.handle, self.exact.data_ptr(), self.exact_flags.data_ptr())
            centres = torch.from_numpy(rng.integers(lo, hi + 1, size=(n, 2)).astype(np.int32)).to(self.device)
            abi.seb_sur_gather(self.handle, worlds[w].data_ptr(), self.exact.data_ptr(), self.world, self.world,
                               centres.data_ptr(), n, off)
            off += n
        return worlds

    def train_step(self, batch, lr):
        self.step += 1
        abi.seb_sur_set_stream(self.handle, self._stream())
        abi.seb_sur_train_step(self.handle, batch, lr, self.step, self.loss.data_ptr())

    def train(self, n_patches, batch=256, lr=2e-3, seed=1000, log_every=0):
        rng = np.random.default_rng(seed)
        steps = (n_patches + batch - 1) // batch
        return self.train_steps(rng, 0, steps, steps, batch, lr, log_every)

    def train_steps(self, rng, first, count, total, batch=256, lr=2e-3, log_every=0):
        """Steps first .. first + count - 1 of a run of `total` steps (cosine learning-rate
        schedule over the run), drawing terrain and patches from `rng`.  A run split into calls,
        or resumed from a checkpoint with the generator state restored, repeats the same steps."""
        losses = []
        for i in range(first, first + count):
            cur_lr = lr * 0.5 * (1 + math.cos(math.pi * i / total))  # cosine schedule
            self.make_batch(rng, batch)
            self.train_step(batch, cur_lr)
            if log_every and (i % log_every == 0 or i == total - 1):
                losses.append((i, float(self.loss.item())))
        return losses

    def infer(self, elev, step=0.04, radius=3, exact_fallback=True):
        """elev [ny][nx] FP32 on the device -> (out [5][K][ny][nx], flags [K][ny][nx], mask [ny][nx])."""
        p = self.params
        if tuple(elev.shape) != (p.ny, p.nx) or elev.dtype != torch.float32 or not elev.is_contiguous():
            raise ValueError(f"elevation must be contiguous float32 ({p.ny}, {p.nx})")
        out = torch.empty((5, p.n_yaw, p.ny, p.nx), dtype=torch.float32, device=self.device)
        fl = torch.empty((p.n_yaw, p.ny, p.nx), dtype=torch.uint8, device=self.device)
        mask = torch.empty((p.ny, p.nx), dtype=torch.uint8, device=self.device)
        self.infer_into(elev, out, fl, mask, step, radius, exact_fallback)
        return out, fl, mask

    def infer_into(self, elev, out, fl, mask, step=0.04, radius=3, exact_fallback=True):
        abi.seb_sur_set_stream(self.handle, self._stream())
        abi.seb_sur_infer(self.handle, elev.data_ptr(), step, radius, 1 if exact_fallback else 0, out.data_ptr(),
                          fl.data_ptr(), mask.data_ptr())

    def state_dict(self):
        """Checkpoint through the C ABI (seb_sur_save: master weights, Adam moments, BF16 weights
        and the Adam step)."""
        abi.seb_sur_set_stream(self.handle, self._stream())
        return {"image": abi.seb_sur_save(self.handle), "step": self.step}

    def load_state_dict(self, sd):
        abi.seb_sur_set_stream(self.handle, self._stream())
        abi.seb_sur_load(self.handle, sd["image"])
        self.step = abi.seb_sur_step(self.handle)
        if self.step != int(sd["step"]):
            raise ValueError("checkpoint step and image disagree")

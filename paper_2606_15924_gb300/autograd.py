"""Differentiable sparse rendering: a torch.autograd.Function around the C-ABI
calls.

``render_sampled(params, raster)`` returns the colours [P, 3] of the sampled
pixels described by ``raster`` (a ``SampledRaster``: camera, active tiles and
per-tile pixel lists).  Its backward calls ``backward_sampled``, which replays
each pixel's compositing in reverse from the stored final transmittance and
last splat index, so no per-(pixel, splat) transmittance is kept between the
passes.  Gradients flow to means, log_scales, quats, opacity_logits and sh.
"""
from __future__ import annotations

import torch

from . import binding as B
from .config import TILE


class SampledRaster:
    """Camera + sampled pixel set + the buffers one forward/backward needs.

    The pixel set is given as device tensors in the select_tiles layout
    (active_tiles [A] ascending, tile_rank [T], pix_off [A+1], pix_idx [P]),
    e.g. straight from ``binding.select_tiles`` or ``SampledRaster.from_tiles``.
    """

    def __init__(self, cam: dict, n_gaussians: int, active_tiles, n_active, tile_rank, pix_off, pix_idx,
                 n_pix: int, capacity: int | None = None, bg=(0.0, 0.0, 0.0), sh_degree: int = 3):
        self.cam = cam
        self.ccam = B.camera(cam)
        self.n = int(n_gaussians)
        self.active_tiles, self.n_active, self.tile_rank = active_tiles, n_active, tile_rank
        self.pix_off, self.pix_idx = pix_off, pix_idx
        self.n_active_max = int(active_tiles.shape[0])
        self.n_pix = int(n_pix)
        # sampled pixels (read once from the device; pix_idx may be longer)
        self.P = int(pix_off[int(n_active.reshape(-1)[0].item())].item())
        self.bg, self.sh_degree = tuple(bg), sh_degree
        dev = active_tiles.device
        n = self.n
        self.proj = dict(xy=torch.zeros(n, 2, device=dev), conic_opac=torch.zeros(n, 4, device=dev),
                         rgb=torch.zeros(n, 3, device=dev), depth=torch.zeros(n, device=dev),
                         radius=torch.zeros(n, dtype=torch.int32, device=dev))
        self.ranges = torch.zeros(max(self.n_active_max, 1), 2, dtype=torch.int32, device=dev)
        self.n_isect = torch.zeros(1, dtype=torch.int64, device=dev)
        self.capacity = int(capacity) if capacity is not None else 0
        self.ws_bin = None
        self.vals = None
        self.T_final = torch.zeros(max(int(pix_idx.shape[0]), 1), device=dev)
        self.n_last = torch.zeros(max(int(pix_idx.shape[0]), 1), dtype=torch.int32, device=dev)
        self.grad2d = torch.zeros(n, 12, device=dev)
        self.touched = torch.zeros(n, dtype=torch.uint8, device=dev)

    @staticmethod
    def from_tiles(cam: dict, n_gaussians: int, tiles, device="cuda", **kw):
        """Every pixel of the given tiles (ids, any order)."""
        W, H = int(cam["width"]), int(cam["height"])
        tx_n = (W + TILE - 1) // TILE
        T = tx_n * ((H + TILE - 1) // TILE)
        tiles = sorted(set(int(t) for t in tiles))
        rank = torch.full((T,), -1, dtype=torch.int32)
        off, idx = [0], []
        for r, t in enumerate(tiles):
            rank[t] = r
            tx, ty = t % tx_n, t // tx_n
            for l in range(TILE * TILE):
                if tx * TILE + l % TILE < W and ty * TILE + l // TILE < H:
                    idx.append(l)
            off.append(len(idx))
        dev = torch.device(device)
        return SampledRaster(cam, n_gaussians, torch.tensor(tiles, dtype=torch.int32, device=dev),
                             torch.tensor([len(tiles)], dtype=torch.int32, device=dev), rank.to(dev),
                             torch.tensor(off, dtype=torch.int32, device=dev),
                             torch.tensor(idx, dtype=torch.uint8, device=dev), TILE * TILE, **kw)

    def pixel_coords(self) -> torch.Tensor:
        """[P, 2] integer (x, y) of the sampled pixels, in output order."""
        A = int(self.n_active.item())
        off = self.pix_off[:A + 1].long()
        tiles = torch.repeat_interleave(self.active_tiles[:A].long(), off[1:] - off[:-1])
        l = self.pix_idx[:int(off[-1])].long()
        tx_n = (int(self.cam["width"]) + TILE - 1) // TILE
        return torch.stack([(tiles % tx_n) * TILE + l % TILE, (tiles // tx_n) * TILE + l // TILE], 1)

    def _ensure_bins(self):
        if self.capacity > 0 and self.vals is not None:
            return
        dev = self.active_tiles.device
        if self.capacity == 0:  # exact pair count (one synchronising query)
            ws = torch.empty(B.bin_tiles_workspace_size(self.n, 0, self.n_active_max), dtype=torch.uint8,
                             device=dev)
            B.bin_tiles(self.proj, self.n, self.ccam, self.tile_rank, self.n_active_max, ws, 0, None, None,
                        self.ranges, self.n_isect)
            self.capacity = int(self.n_isect.item()) + 1024
        self.ws_bin = torch.empty(B.bin_tiles_workspace_size(self.n, self.capacity, self.n_active_max),
                                  dtype=torch.uint8, device=dev)
        self.vals = torch.zeros(self.capacity, dtype=torch.int32, device=dev)

    def forward_buffers(self, params: dict) -> torch.Tensor:
        """project -> bin -> render; returns rgb [P, 3] (new tensor)."""
        B.project_gaussians(params, self.ccam, self.tile_rank, self.proj, self.sh_degree)
        self._ensure_bins()
        B.bin_tiles(self.proj, self.n, self.ccam, self.tile_rank, self.n_active_max, self.ws_bin, self.capacity,
                    self.vals, None, self.ranges, self.n_isect)
        need = int(self.n_isect.item())
        if need > self.capacity:  # the Gaussians moved: grow and bin again
            self.capacity = int(need * 1.25) + 1024
            self.vals = None
            self._ensure_bins()
            B.bin_tiles(self.proj, self.n, self.ccam, self.tile_rank, self.n_active_max, self.ws_bin,
                        self.capacity, self.vals, None, self.ranges, self.n_isect)
        rgb = torch.zeros(max(int(self.pix_idx.shape[0]), 1), 3, device=self.active_tiles.device)
        B.render_sampled(self.proj, self.ranges, self.vals, self.active_tiles, self.n_active, self.n_active_max,
                         self.pix_off, self.pix_idx, self.n_pix, self.ccam, self.bg, rgb, self.T_final, self.n_last)
        return rgb[:self.P]


class _RenderSampled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, raster):
        params = dict(means=means.contiguous(), log_scales=log_scales.contiguous(), quats=quats.contiguous(),
                      opacity_logits=opacity_logits.contiguous(), sh=sh.contiguous())
        rgb = raster.forward_buffers(params)
        ctx.raster = raster
        ctx.save_for_backward(params["means"], params["log_scales"], params["quats"], params["opacity_logits"],
                              params["sh"])
        return rgb

    @staticmethod
    def backward(ctx, dL_drgb):
        raster = ctx.raster
        means, log_scales, quats, opacity_logits, sh = ctx.saved_tensors
        params = dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=opacity_logits, sh=sh)
        grads = {k: torch.empty_like(v) for k, v in params.items()}
        g = torch.zeros(max(int(raster.pix_idx.shape[0]), 1), 3, device=means.device)
        g[:raster.P] = dL_drgb
        B.backward_sampled(params, raster.ccam, raster.proj, raster.ranges, raster.vals, raster.active_tiles,
                           raster.n_active, raster.n_active_max, raster.pix_off, raster.pix_idx, raster.n_pix,
                           raster.bg, raster.T_final, raster.n_last, g, raster.grad2d, grads, raster.touched,
                           write_untouched=True, sh_degree=raster.sh_degree)
        return grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logits"], grads["sh"], None


def render_sampled(params: dict, raster: SampledRaster) -> torch.Tensor:
    """Differentiable colours [P, 3] of the sampled pixels."""
    return _RenderSampled.apply(params["means"], params["log_scales"], params["quats"], params["opacity_logits"],
                                params["sh"], raster)

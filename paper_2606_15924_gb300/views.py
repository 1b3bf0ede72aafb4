"""Adaptive view budget and geometry-aware view sampling (Sec. 3.4; App. A).

At iteration t the method first sets its view budget K_t and tile pixel rate
r_tile from the error trend (App. A, Eqs. 15-16: host arithmetic, Alg. 1 step
1), then draws K_t views (Alg. 1 step 2): the anchor with the largest mean
error (Eq. 5) and K_t - 1 others weighted by camera proximity and viewing
direction (Eq. 6), without replacement from a view stack.  The mean errors
and the draw run on the GPU (``view_error_sums``, ``sample_views``); the
schedule needs the mean over all views on the host, which is one small copy
of V integers per iteration.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B
from .config import ScheduleConfig

ERR_SCALE = float(2 ** 24)  # view_error_sums counts E * 2^24


def sampling_schedule(t: int, E_t: float, E_init: float, sched: ScheduleConfig | None = None,
                      eps: float = 1e-8) -> tuple[int, float]:
    """(K_t, r_tile) at iteration t from the current and initial mean view
    errors (App. A, Eqs. 15-16).

    The error ratio r = clip(E_t / (E_init + eps), 0, 1) is bent by
    phi = sin(pi/2 sqrt(r)); the progress coefficient is the appendix's
    rho = 1 - clip(t / tau_until, 0, 1), which is 1 at the start and 0 once
    densification ends.  With g = 1 - rho phi the pixel rate moves from
    lambda / K_max (g = 0: early, high error) to lambda / K_min (g = 1) and
    the budget from K_max towards K_min + (K_max - K_min) e^-alpha; K_t rounds
    halves up."""
    s = sched or ScheduleConfig()
    ratio = min(max(E_t / (E_init + eps), 0.0), 1.0)
    phi = math.sin(0.5 * math.pi * math.sqrt(ratio))
    rho = 1.0 - min(max(t / s.tau_until, 0.0), 1.0)
    g = 1.0 - rho * phi
    r_lo, r_hi = s.lam / s.K_max, s.lam / s.K_min
    r_tile = r_lo + (r_hi - r_lo) * g
    K = int(math.floor(s.K_min + (s.K_max - s.K_min) * math.exp(-s.alpha * g) + 0.5))
    return K, r_tile


def pixels_per_tile(r_tile: float) -> int:
    """Sampled pixels of a full 16 x 16 tile at rate r_tile (1 to 256)."""
    return max(1, min(256, int(math.floor(r_tile * 256.0 + 0.5))))


def camera_pose(cam: dict) -> tuple[np.ndarray, np.ndarray]:
    """Camera centre -R^T t and unit forward axis of a world-to-camera matrix."""
    M = np.asarray(cam["viewmat"], dtype=np.float64).reshape(4, 4)
    R, t = M[:3, :3], M[:3, 3]
    f = R[2]
    return -R.T @ t, f / np.linalg.norm(f)


class ViewSampler:
    """Per-iteration view draw over a fixed set of V cameras (Alg. 1 step 2).

    lambda_d and lambda_theta weight camera distance and viewing direction in
    Eq. 6; the paper leaves both open.  By default lambda_d is 2 / (the median
    distance between camera centres), which makes the weight scale-free, and
    lambda_theta is 2.  The stack starts full and lives on the device."""

    def __init__(self, cams: list, lambda_d: float | None = None, lambda_theta: float = 2.0, seed: int = 0,
                 device="cuda"):
        V = len(cams)
        if not 1 <= V <= 8192:
            raise ValueError("1 to 8192 views")
        self.V = V
        if lambda_d is None:
            c = np.stack([camera_pose(cm)[0] for cm in cams])
            d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))[np.triu_indices(V, 1)]
            med = float(np.median(d)) if d.size else 0.0
            lambda_d = 2.0 / med if med > 0.0 else 0.0
        self.lambda_d, self.lambda_theta, self.seed = float(lambda_d), float(lambda_theta), int(seed)
        self.cams = B.camera_array(cams, device)
        self.stack = torch.ones(V, dtype=torch.uint8, device=device)
        self.sums = torch.zeros(V, dtype=torch.int64, device=device)
        self.views = torch.zeros(V, dtype=torch.int32, device=device)
        self.n_pix = int(cams[0]["width"]) * int(cams[0]["height"])

    def error_sums(self, err_maps: torch.Tensor) -> torch.Tensor:
        """Exact per-view totals of the error maps [V,H,W] (fp16 bits)."""
        B.view_error_sums(err_maps, self.sums)
        return self.sums

    def mean_errors(self) -> np.ndarray:
        """Mean error of every view (Eq. 5's E-bar), on the host."""
        return self.sums.cpu().numpy().astype(np.float64) / ERR_SCALE / self.n_pix

    def draw(self, k: int, it: int) -> torch.Tensor:
        """k views for iteration it from the current error sums: device int32
        [k], the anchor first."""
        B.sample_views(self.sums, self.cams, k, self.lambda_d, self.lambda_theta, self.seed, it, self.stack,
                       self.views)
        return self.views[:k]


class ScheduledTrainer:
    """Alg. 1 steps 1-2 in front of the multi-view step (steps 3-10).

    Every view of the pool keeps its error and age maps resident, the error
    maps as slices of one [V,H,W] tensor.  At construction each view's map is
    set by one dense evaluation (Sec. 3.3), which fixes E_init.  Iteration t
    then computes every view's error total on the GPU, reads the V totals
    back for the schedule (K_t, r_tile), draws K_t views (anchor first), and
    runs one step of the persistent multi-view trainer over them with
    round(256 r_tile) pixels per tile.  K_t is capped at 16 views per step.
    All views must share one image size."""

    def __init__(self, params: dict, cams: list, targets: list, tile_fraction: float = 0.2, cfg=None, seed: int = 0,
                 lambda_d: float | None = None, lambda_theta: float = 2.0, **kw):
        from .batched import MultiViewTrainer
        from .config import Config
        self.cfg = cfg or Config()
        s = self.cfg.schedule
        V = len(cams)
        W, H = int(cams[0]["width"]), int(cams[0]["height"])
        if any(int(c["width"]) != W or int(c["height"]) != H for c in cams):
            raise ValueError("all views need one image size")
        # pool buffers sized for the largest pixel rate, lambda / K_min
        cap = pixels_per_tile(s.lam / s.K_min)
        self.mv = MultiViewTrainer(params, cams, targets, [tile_fraction] * V, pixel_rate=(cap + 0.5) / 256.0,
                                   cfg=self.cfg, seed=seed, max_active=min(s.K_max, V, 16), **kw)
        dev = params["means"].device
        self.err_maps = torch.zeros(V, H, W, dtype=torch.int16, device=dev)
        for k, v in enumerate(self.mv.pool):
            v.err_map = self.err_maps[k]
            v.init_error_map()
        self.sampler = ViewSampler(cams, lambda_d=lambda_d, lambda_theta=lambda_theta, seed=seed, device=dev)
        self.sched = s
        self.E_init = None
        self.t = 0
        self.history = []

    def step(self) -> dict:
        self.sampler.error_sums(self.err_maps)
        E_t = float(self.sampler.mean_errors().mean())
        if self.E_init is None:
            self.E_init = E_t
        K, r = sampling_schedule(self.t, E_t, self.E_init, self.sched)
        K = max(1, min(K, self.mv.max_active))
        ids = self.sampler.draw(K, self.t).cpu().tolist()
        n_pix = pixels_per_tile(r)
        self.mv.set_views(ids, n_pix)
        self.mv.step()
        rec = dict(t=self.t, K=K, r_tile=r, n_pix=n_pix, views=ids, E_t=E_t)
        self.history.append(rec)
        self.t += 1
        return rec

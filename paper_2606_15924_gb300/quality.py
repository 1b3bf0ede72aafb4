"""Sampled against dense training at equal quality.

The sparse path only pays off if it reaches the quality of plain dense
training in less time.  ``compare`` trains the same initial Gaussians towards
the same target twice, with the dense path (every tile, every pixel) and with
the sampled path (error-guided tiles and pixels, Sec. 3.5), both as captured
graph replays of the same library, and records PSNR against the target over
device time.  Evaluation renders run between timed segments and are not
counted.

Scene recipe (the paper's datasets are not available): a seeded ground-truth
cloud renders the target; training starts from that cloud with perturbed
means (sigma 0.02 x extent), log-scales (+N(0, 0.3)), re-drawn SH
coefficients and opacities.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import scenes
from .pipeline import Trainer


def perturbed_init(gt: dict, extent: float, seed: int = scenes.SEED_NOISE) -> dict:
    rng = np.random.default_rng(seed)
    n = gt["means"].shape[0]
    return dict(means=(gt["means"] + rng.normal(0.0, 0.02 * extent, size=(n, 3))).astype(np.float32),
                log_scales=(gt["log_scales"] + rng.normal(0.0, 0.3, size=(n, 3))).astype(np.float32),
                quats=gt["quats"].copy(),
                opacity_logits=rng.normal(size=n).astype(np.float32),
                sh=rng.normal(0.0, 0.2, size=gt["sh"].shape).astype(np.float32))


class Evaluator:
    """Full-image PSNR of the current Gaussians against the target, through one
    dense render-only pass of the library (buffers kept between calls)."""

    def __init__(self, params: dict, cam: dict, target: torch.Tensor):
        self.d = Trainer(params, cam, target, dense=True, train=False)
        self.d.forward()
        xy = self.d.pixel_coords()
        self.P = xy.shape[0]
        self.ref = target[xy[:, 1], xy[:, 0]].contiguous()

    def psnr(self) -> float:
        self.d.forward()
        mse = torch.mean((self.d.rgb[:self.P].clamp(0, 1) - self.ref) ** 2).item()
        return float(10.0 * math.log10(1.0 / max(mse, 1e-12)))


def train_curve(tr: Trainer, ev: Evaluator, max_iters: int, eval_every: int, stop_psnr: float | None = None,
                max_ms: float | None = None) -> dict:
    """Replays tr's graph in segments of eval_every iterations; returns the
    curve [(iterations, device ms, psnr)]."""
    curve = [(0, 0.0, ev.psnr())]
    ms, it = 0.0, 0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while it < max_iters:
        k = min(eval_every, max_iters - it)
        torch.cuda.synchronize()
        a.record()
        for _ in range(k):
            tr.replay()
        b.record()
        b.synchronize()
        ms += a.elapsed_time(b)
        it += k
        p = ev.psnr()
        curve.append((it, ms, p))
        if stop_psnr is not None and p >= stop_psnr:
            break
        if max_ms is not None and ms >= max_ms:
            break
    return dict(curve=curve, iters=it, ms=ms, psnr=curve[-1][2], iters_per_s=it / (ms * 1e-3) if ms else 0.0)


def time_to(curve: list, psnr: float):
    """Device ms at which a curve first reaches psnr (linear between points),
    or None."""
    prev = curve[0]
    if prev[2] >= psnr:
        return 0.0
    for pt in curve[1:]:
        if pt[2] >= psnr:
            f = (psnr - prev[2]) / max(pt[2] - prev[2], 1e-12)
            return prev[1] + f * (pt[1] - prev[1])
        prev = pt
    return None


def compare(device, n: int = 500_000, width: int = 1280, height: int = 720, distance: float = 15.0,
            extent: float = 5.0, dense_iters: int = 2000, eval_every: int = 250, tile_fraction: float = 0.2,
            pixel_rate: float = 1.0 / 3.0, time_cap: float = 1.5, settings=None) -> dict:
    """Dense for dense_iters iterations; sampled until it is within 0.1 dB of
    the dense final PSNR or has used time_cap x the dense device time.
    settings: list of (tile_fraction, pixel_rate) for the sampled runs (one
    dense run serves them all); default the single given pair."""
    if settings is None:
        settings = [(tile_fraction, pixel_rate)]
    cam = scenes.look_at((0.0, 0.0, -distance), width=width, height=height)
    gt = scenes.gaussians(n, seed=scenes.SEED_TARGET, extent=extent)
    gt_d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in gt.items()}
    dummy = torch.zeros(height, width, 3, device=device)
    target = Trainer(gt_d, cam, dummy, dense=True, train=False).render_image().contiguous()
    del gt_d
    init = perturbed_init(gt, extent)
    out = {"workload": f"{n} Gaussians, {width}x{height}, perturbed ground truth"}
    runs = {}
    for name, (frac, rate) in [("dense", (1.0, 1.0))] + [(f"sampled_{f:g}_{r:.3g}", (f, r)) for f, r in settings]:
        params = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in init.items()}
        dense = name == "dense"
        tr = Trainer(params, cam, target, tile_fraction=frac, pixel_rate=rate, dense=dense)
        ev = Evaluator(params, cam, target)
        t_init = 0.0
        if not dense:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            tr.init_error_map()
            b.record()
            b.synchronize()
            t_init = a.elapsed_time(b)
        tr.capture()
        # the capture's warm-up step trained once: count it
        if dense:
            r = train_curve(tr, ev, dense_iters, eval_every)
        else:
            goal = runs["dense"]["psnr"] - 0.1
            r = train_curve(tr, ev, 10 ** 7, eval_every * 2, stop_psnr=goal,
                            max_ms=time_cap * runs["dense"]["ms"])
            r["error_map_init_ms"] = t_init
        r["overflowed"] = tr.overflowed()
        if not dense:
            r.update(tile_fraction=frac, pixel_rate=rate)
        runs[name] = r
        del tr, ev, params
        torch.cuda.empty_cache()
    d = runs.pop("dense")
    goal = d["psnr"] - 0.1
    t_d = time_to(d["curve"], goal)
    out.update(dense=d, psnr_goal=goal, sampled={})
    for name, s in runs.items():
        t_s = time_to(s["curve"], goal)
        s.update(iters_per_s_ratio=s["iters_per_s"] / d["iters_per_s"], reached=t_s is not None,
                 time_to_goal_ms=None if t_s is None else t_s + s.get("error_map_init_ms", 0.0),
                 dense_time_to_goal_ms=t_d)
        if t_s is not None:
            s["time_speedup"] = t_d / s["time_to_goal_ms"]
        out["sampled"][name] = s
    return out

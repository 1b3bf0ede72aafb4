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
from .pipeline import Trainer, as_geo_rows


def jittered_init(gt: dict, extent: float, seed: int = scenes.SEED_NOISE, mean_sigma: float = 0.004,
                  scale_sigma: float = 0.1, opacity_sigma: float = 0.5, sh_sigma: float = 0.1) -> dict:
    """The ground truth with every parameter moved by Gaussian noise: means
    by N(0, (mean_sigma extent)^2), log-scales by N(0, scale_sigma^2), opacity
    logits by N(0, opacity_sigma^2), SH coefficients by N(0, sh_sigma^2) (a
    partly fitted scene, in place of one whose colours are drawn anew)."""
    rng = np.random.default_rng(seed)
    n = gt["means"].shape[0]
    return dict(means=(gt["means"] + rng.normal(0.0, mean_sigma * extent, size=(n, 3))).astype(np.float32),
                log_scales=(gt["log_scales"] + rng.normal(0.0, scale_sigma, size=(n, 3))).astype(np.float32),
                quats=gt["quats"].copy(),
                opacity_logits=(gt["opacity_logits"] + rng.normal(0.0, opacity_sigma, size=n)).astype(np.float32),
                sh=(gt["sh"] + rng.normal(0.0, sh_sigma, size=gt["sh"].shape)).astype(np.float32))


def perturbed_init(gt: dict, extent: float, seed: int = scenes.SEED_NOISE, mean_sigma: float = 0.02) -> dict:
    """The ground truth with means moved by N(0, (mean_sigma extent)^2),
    log-scales by N(0, 0.3^2), and opacities and SH coefficients re-drawn."""
    rng = np.random.default_rng(seed)
    n = gt["means"].shape[0]
    return dict(means=(gt["means"] + rng.normal(0.0, mean_sigma * extent, size=(n, 3))).astype(np.float32),
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
        return prev[1]
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
        params = as_geo_rows({k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in init.items()})
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


# ---------------------------------------------------------------------------
# several views, held-out evaluation
# ---------------------------------------------------------------------------

class ViewCycle:
    """Training over a set of views one view per iteration, in the order of a
    seeded permutation renewed every pass (as plain 3DGS training draws its
    views).  Every view has its own trainer and captured step; all of them
    share the Gaussians and the optimiser state (moments, step counter).
    dense=True gives the library's plain path (every tile, every pixel);
    otherwise each step samples tile_fraction of the tiles and pixel_rate of
    their pixels, guided by the view's own error and age maps."""

    def __init__(self, params: dict, cams: list, targets: list, dense: bool, tile_fraction: float = 1.0,
                 pixel_rate: float = 1.0, seed: int = 0):
        self.trs = []
        for k, (cam, tgt) in enumerate(zip(cams, targets)):
            self.trs.append(Trainer(params, cam, tgt, tile_fraction=tile_fraction, pixel_rate=pixel_rate,
                                    dense=dense, seed=seed, view=k, share=self.trs[0] if self.trs else None))
        self.params = params
        self.dense = dense
        self.rng = np.random.default_rng(seed)
        self.order = []

    def init_error_maps(self):
        """Every view's E_v from one dense evaluation (Sec. 3.3)."""
        for tr in self.trs:
            tr.init_error_map()

    def capture(self):
        """One captured step per view.  Each capture's warm-up step is undone:
        the Gaussians and the optimiser state are restored afterwards."""
        t0 = self.trs[0]
        keep = [{k: v.clone() for k, v in d.items()} for d in (self.params, t0.m, t0.v)]
        step, it = t0.step_dev.clone(), t0.it_dev.clone()
        for tr in self.trs:
            tr.capture(overlap=True)
        for d, saved in zip((self.params, t0.m, t0.v), keep):
            for k in d:
                d[k].copy_(saved[k])
        t0.step_dev.copy_(step)
        t0.it_dev.copy_(it)
        torch.cuda.synchronize()

    def replay(self):
        if not self.order:
            self.order = list(self.rng.permutation(len(self.trs)))
        self.trs[self.order.pop()].replay()

    def overflowed(self) -> bool:
        return any(tr.overflowed() for tr in self.trs)


class HeldOutEvaluator:
    """Mean PSNR over held-out views, each over its foreground pixels (where
    the ground truth's final transmittance is below 1/2), from one dense
    render-only pass of the library per view."""

    def __init__(self, params: dict, cams: list, targets: list, masks: list):
        self.views = []
        for cam, tgt, mask in zip(cams, targets, masks):
            d = Trainer(params, cam, tgt, dense=True, train=False)
            d.forward()
            xy = d.pixel_coords()
            keep = mask[xy[:, 1], xy[:, 0]]
            self.views.append((d, keep, tgt[xy[:, 1], xy[:, 0]][keep].contiguous()))

    def psnr(self) -> float:
        out = []
        for d, keep, ref in self.views:
            d.forward()
            mse = torch.mean((d.rgb[:keep.shape[0]][keep].clamp(0, 1) - ref) ** 2).item()
            out.append(10.0 * math.log10(1.0 / max(mse, 1e-12)))
        return float(np.mean(out))


def _gt_views(gt_d: dict, cams: list, noise: float, seed: int):
    """Targets (renders of the ground truth + N(0, noise^2)) and foreground
    masks (ground-truth final transmittance < 1/2) of every view."""
    gen = torch.Generator().manual_seed(seed)
    targets, masks = [], []
    for cam in cams:
        H, W = int(cam["height"]), int(cam["width"])
        d = Trainer(gt_d, cam, torch.zeros(H, W, 3, device=gt_d["means"].device), dense=True, train=False)
        d.forward()
        img = d.scatter_image(d.rgb)
        Timg = d.scatter_image(d.T_final[:, None])[..., 0]
        targets.append((img + torch.randn(H, W, 3, generator=gen).to(img.device) * noise).contiguous())
        masks.append(Timg < 0.5)
    return targets, masks


def _run_curve(step, ev, max_iters: int, eval_every: int, stop_psnr=None, max_ms=None, extra_ms: float = 0.0):
    curve = [(0, extra_ms, ev.psnr())]
    ms, it = extra_ms, 0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while it < max_iters:
        k = min(eval_every, max_iters - it)
        torch.cuda.synchronize()
        a.record()
        for _ in range(k):
            step()
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
    return dict(curve=curve, iters=it, ms=ms, psnr=curve[-1][2],
                iters_per_s=it / ((ms - extra_ms) * 1e-3) if ms > extra_ms else 0.0)


def compare_views(device, n: int = 500_000, width: int = 1280, height: int = 720, distance: float = 15.0,
                  extent: float = 5.0, n_views: int = 64, hold_every: int = 8, noise: float = 0.01,
                  dense_iters: int = 3000, eval_every: int = 250, time_cap: float = 1.5, settings=None,
                  scheduled: bool = True, scheduled_fraction: float = 1.0, mean_sigma: float = 0.02,
                  init: str = "perturbed") -> dict:
    """Dense against sampled training on an orbit of views with every
    hold_every-th view held out, at equal held-out PSNR (device time).

    The ground-truth cloud renders the targets (+ N(0, noise^2)); training
    starts from it perturbed (``perturbed_init``).  The dense run trains
    dense_iters iterations, one view each (``ViewCycle``); each sampled
    setting (tile_fraction, pixel_rate) trains the same way on sampled tiles
    and pixels until its held-out PSNR is within 0.1 dB of the dense run's
    final value, or it has used time_cap x the dense device time.  With
    scheduled=True the paper's multi-view iteration runs too: the adaptive
    view budget and pixel rate and the geometry-aware view draw
    (``views.ScheduledTrainer``, Sec. 3.4, App. A) over the training views,
    on scheduled_fraction of the tiles."""
    from .views import ScheduledTrainer
    if settings is None:
        settings = [(1.0, 0.1), (1.0, 1.0 / 3.0)]
    cams = scenes.orbit(n_views, distance, width, height)
    held = [k for k in range(n_views) if k % hold_every == hold_every // 2]
    train = [k for k in range(n_views) if k not in held]
    gt = scenes.gaussians(n, seed=scenes.SEED_TARGET, extent=extent)
    gt_d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in gt.items()}
    targets, masks = _gt_views(gt_d, cams, noise, scenes.SEED_NOISE)
    del gt_d
    init_kind = init
    if init_kind == "jitter":
        init = jittered_init(gt, extent, mean_sigma=mean_sigma)
    else:
        init = perturbed_init(gt, extent, mean_sigma=mean_sigma)
    fg = float(np.mean([m.float().mean().item() for m in masks]))
    out = {"workload": f"{n} Gaussians, {len(train)} training and {len(held)} held-out views of a {n_views}-view "
                       f"orbit at {width}x{height}, {init_kind} ground truth (means sigma {mean_sigma:g} x extent), "
                       f"targets + N(0, {noise:g}^2)",
           "psnr": f"mean over the held-out views of the PSNR over foreground pixels (ground-truth T < 1/2; "
                   f"{100 * fg:.0f}% of the pixels)"}
    runs = {}
    arms = [("dense", None)] + [(f"sampled_{f:g}_{r:.3g}", (f, r)) for f, r in settings]
    if scheduled:
        arms.append((f"scheduled_{scheduled_fraction:g}", "scheduled"))
    for name, setting in arms:
        params = as_geo_rows({k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in init.items()})
        ev = HeldOutEvaluator(params, [cams[k] for k in held], [targets[k] for k in held], [masks[k] for k in held])
        t_init = 0.0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if setting == "scheduled":
            tr = ScheduledTrainer(params, [cams[k] for k in train], [targets[k] for k in train],
                                  tile_fraction=scheduled_fraction)
            # the dense evaluation of every view that set E_init, timed again on the same Gaussians
            a.record()
            for v in tr.mv.pool:
                v.init_error_map()
            b.record()
            b.synchronize()
            t_init = a.elapsed_time(b)
            step = tr.step
        else:
            dense = setting is None
            f, r = (1.0, 1.0) if dense else setting
            tr = ViewCycle(params, [cams[k] for k in train], [targets[k] for k in train], dense, f, r)
            tr.capture()
            if not dense:
                a.record()
                tr.init_error_maps()
                b.record()
                b.synchronize()
                t_init = a.elapsed_time(b)
            step = tr.replay
        if name == "dense":
            res = _run_curve(step, ev, dense_iters, eval_every)
        else:
            goal = runs["dense"]["psnr"] - 0.1
            res = _run_curve(step, ev, 10 ** 7, eval_every, stop_psnr=goal, max_ms=time_cap * runs["dense"]["ms"],
                             extra_ms=t_init)
            res["error_map_init_ms"] = t_init
        res["overflowed"] = tr.mv.overflowed() if setting == "scheduled" else tr.overflowed()
        if setting == "scheduled":
            hist = tr.history
            res["views_per_iter"] = float(np.mean([h["K"] for h in hist])) if hist else 0.0
            res["pixels_per_tile"] = [hist[0]["n_pix"], hist[-1]["n_pix"]] if hist else []
        elif setting is not None:
            res.update(tile_fraction=setting[0], pixel_rate=setting[1])
        runs[name] = res
        del tr, ev, params
        torch.cuda.empty_cache()
    d = runs.pop("dense")
    goal = d["psnr"] - 0.1
    t_d = time_to(d["curve"], goal)
    out.update(dense=d, psnr_goal=goal, sampled={})
    for name, s in runs.items():
        t_s = time_to(s["curve"], goal)
        s.update(iters_per_s_ratio=s["iters_per_s"] / d["iters_per_s"], reached=t_s is not None,
                 time_to_goal_ms=t_s, dense_time_to_goal_ms=t_d)
        if t_s is not None and t_s > 0:
            s["time_speedup"] = t_d / t_s
        out["sampled"][name] = s
    return out

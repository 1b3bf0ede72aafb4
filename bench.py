"""Throughput of the TurboGS sparse-sampled training step on one GB300.

Workload (the sparse-training-step configuration): 500k Gaussians (means
uniform in [-5,5]^3, log-scales N(-3.5,0.5), unit quaternions, opacity logits
N(0,1), SH degree 3 ~ N(0,0.2)), one 1280x720 pinhole view (fov 60 deg, distance
15), a target rendered from a second seeded Gaussian set, an error map from the
dense render of the initial Gaussians.  A step is one full training iteration
of the sampled path: tile selection + pixel sampling, projection, binning,
sparse render, fused L1 + sparse-NCC loss with error/age updates, sparse
backward, hybrid LM/Adam update.  The same library's dense path (every tile,
every pixel) is measured beside it.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GAUSS = 500_000
WIDTH, HEIGHT = 1280, 720
DISTANCE = 15.0
EXTENT = 5.0
TILE_FRACTION = 0.2
PIXEL_RATE = 1.0 / 3.0
METRIC = "train iters/s & sampled fwd+bwd Mpix/s vs dense path, 1 GB300, same PSNR"
L2_FLUSH_BYTES = 256 << 20


def workload_config(frac=TILE_FRACTION, rate=PIXEL_RATE):
    return {"workload": "sparse training step: 500k Gaussians, 1280x720 view, "
                        f"{round(frac * 100)}% of 16x16 tiles, pixel rate {rate:.3f}",
            "gaussians": N_GAUSS, "width": WIDTH, "height": HEIGHT, "tile_fraction": frac, "pixel_rate": rate,
            "l2": "flushed between timed steps (256 MB write)"}


def sm_count() -> int:
    """Streaming multiprocessors of the current CUDA device."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def alu_peak_tflops(sm_mhz: float) -> float:
    """FP32 peak (FMA = 2 FLOPs) at the given SM clock: SMs x 128 lanes x 2."""
    return sm_count() * 128 * 2 * sm_mhz * 1e6 / 1e12


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class NvmlClocks:
    """SM clock and clock-event reasons read through NVML's C API (ctypes), so
    that a timed region of a few milliseconds still gets samples.  Read-only:
    no setting of the GPU is touched."""
    # nvmlClocksEventReasons bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, gpu_index):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        try:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        v = ctypes.c_uint()
        self.max_mhz = float(v.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(v)) == 0 else None

    def sample(self):
        ct = self.ct
        v, r = ct.c_uint(), ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(v)) != 0:
            return None
        reasons = []
        if self.reasons_fn(self.h, ct.byref(r)) == 0:
            reasons = [nm for bit, nm in self.REASONS.items() if r.value & bit]
        return float(v.value), reasons


class ClockSampler:
    """Clocks during the timed region: NVML every 2 ms in a thread where the
    library loads, else nvidia-smi every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.nvml = None
        self.lines = []
        self.samples = []
        self.stop_flag = threading.Event()

    def start(self):
        try:
            self.nvml = NvmlClocks(self.gpu)
        except OSError:
            self.nvml = None
        if self.nvml is not None:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _poll(self):
        while not self.stop_flag.is_set():
            s = self.nvml.sample()
            if s is not None:
                self.samples.append(s)
            self.stop_flag.wait(0.002)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self.stop_flag.set()
            self.t.join(timeout=5)
            sm = [s[0] for s in self.samples]
            reasons = sorted({r for s in self.samples for r in s[1]})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.nvml.max_mhz,
                    "reasons": reasons, "samples": len(sm), "source": "nvml"}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def build_scene(device):
    import numpy as np
    import torch
    from paper_2606_15924_gb300 import scenes
    from paper_2606_15924_gb300.pipeline import Trainer
    cam = scenes.look_at((0.0, 0.0, -DISTANCE), width=WIDTH, height=HEIGHT, fov_x_deg=60.0)
    gt = scenes.gaussians(N_GAUSS, seed=scenes.SEED_TARGET, extent=EXTENT)
    gt_d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in gt.items()}
    dummy = torch.zeros(HEIGHT, WIDTH, 3, device=device)
    target = Trainer(gt_d, cam, dummy, dense=True, train=False).render_image().contiguous()
    del gt_d
    g = scenes.gaussians(N_GAUSS, seed=scenes.SEED_SCENE, extent=EXTENT)
    return cam, g, target


def make_trainer(g_np, cam, target, dense, frac, rate, device):
    import numpy as np
    import torch
    from paper_2606_15924_gb300.pipeline import Trainer
    from paper_2606_15924_gb300.pipeline import as_geo_rows
    # geometric fields in 64-byte rows (the update of scattered Gaussians then
    # moves whole rows); gradients and moments follow the same layout
    params = as_geo_rows({k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in g_np.items()})
    tr = Trainer(params, cam, target, tile_fraction=frac, pixel_rate=rate, dense=dense)
    tr.init_error_map()
    return tr


def time_replays(tr, steps, flush):
    """Per-step device time of graph replays, L2 flushed between steps."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k)
        ev[k][0].record()
        tr.replay()
        ev[k][1].record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def stage_times_graphs(tr, steps, flush):
    """Mean device time of each stage graph of ``tr`` (events between the
    replays on the launching stream, L2 flushed before each step)."""
    import torch
    if not getattr(tr, "stage_graphs", None):
        tr.capture_stages()
    acc = {n: 0.0 for n, _ in tr.stage_graphs}
    for k in range(steps):
        flush.fill_(k)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(len(tr.stage_graphs) + 1)]
        e[0].record()
        for i, (_, gr) in enumerate(tr.stage_graphs):
            gr.replay()
            e[i + 1].record()
        torch.cuda.synchronize()
        for i, (n, _) in enumerate(tr.stage_graphs):
            acc[n] += e[i].elapsed_time(e[i + 1])
    return {n: acc[n] / steps for n in acc}


def stage_times(tr, steps, flush):
    """Device time of every call of the step: each call is its own captured
    graph, replayed in step order with CUDA events between them on the
    launching stream (L2 flushed before each step); plus the work counts the
    roofline needs."""
    import torch
    if not getattr(tr, "stage_graphs", None):
        tr.capture_stages()
    acc = {n: 0.0 for n, _ in tr.stage_graphs}
    evals = 0
    for k in range(steps):
        flush.fill_(k)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(len(tr.stage_graphs) + 1)]
        e[0].record()
        for i, (_, gr) in enumerate(tr.stage_graphs):
            gr.replay()
            e[i + 1].record()
        torch.cuda.synchronize()
        for i, (n, _) in enumerate(tr.stage_graphs):
            acc[n] += e[i].elapsed_time(e[i + 1])
        A = int(tr.n_active.item())
        P = int(tr.pix_off[A].item())
        evals += int(tr.n_last[:P].sum().item())
    rl = (tr.ranges[:A, 1] - tr.ranges[:A, 0]).float()
    info_tiles = dict(list_mean=float(rl.mean().item()), list_max=int(rl.max().item()),
                      n_last_mean=float(tr.n_last[:P].float().mean().item()), n_last_max=int(tr.n_last[:P].max().item()))
    # the forward tests every splat of a pixel's tile list until the pixel saturates; a pixel can
    # have stopped early only if its T_final is below 0.01 (the stop comes before a splat that
    # takes T below 1e-4, with alpha <= 0.99): such pixels count up to n_last only, the rest the
    # whole list (a lower bound of the alpha tests the method needs)
    npix = (tr.pix_off[1:A + 1] - tr.pix_off[:A]).long()
    L_pix = torch.repeat_interleave(rl, npix)
    maybe = tr.T_final[:P] < 0.01
    walked = float(torch.where(maybe, tr.n_last[:P].float(), L_pix).sum().item())
    maybe_stopped = float(maybe.float().mean().item())
    info = dict(tiles=info_tiles, P=P, A=A, n_isect=int(tr.n_isect.item()), evals_per_step=evals / steps,
                walked_per_step=walked, maybe_stopped=maybe_stopped,
                touched=int(tr.touched.sum().item()) if tr.train else 0,
                visible=int((tr.proj["radius"] > 0).sum().item()))
    return {n: acc[n] / steps for n in acc}, info


# FP32 operations of one alpha evaluation (offset, conic quadratic form,
# exponent scaling, opacity product, clamp) and of one blend (1 - alpha,
# transmittance product, weight, three colour FMAs), FMA = 2; the backward
# replay of one (pixel, splat): alpha again, the transmittance division, the
# colour and alpha adjoints, the conic and centre adjoints (about 45).
FLOPS_ALPHA = 15
FLOPS_BLEND = 10
FLOPS_BWD = 45


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def source_digest(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(stage: str):
    """DRAM bytes per launch of the stage's kernel from the committed ncu
    summary, or None when there is none or the kernel's sources changed since
    it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f).get(stage)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("sources_sha256") != source_digest(rec.get("sources", [])):
        return None
    return rec.get("bytes_per_launch")


# Stages that are one kernel of the library (render_backward also zeroes
# grad2d first); the others chain several small kernels.
SINGLE_KERNEL_STAGES = ("render_sampled", "render_backward", "project_backward", "project_backward_update",
                        "project_gaussians")


def roofline(stage_ms, info, peaks, peak_kind, clocks, tr, dom=None):
    """A stage's kernel against its roof (achieved from its live CUDA-event
    time and its algorithmic work); by default the longest single kernel."""
    if dom is None:
        dom = max((k for k in stage_ms if k in SINGLE_KERNEL_STAGES), key=stage_ms.get)
    t = stage_ms[dom] * 1e-3
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    alu_peak = alu_peak_tflops(sm_mhz)  # TFLOP/s FP32 at the sampled clock
    n = tr.n
    if dom == "render_sampled":
        # an alpha test for every (sampled pixel, list position) walked, a blend up to n_last
        work = (info["walked_per_step"] * FLOPS_ALPHA + info["evals_per_step"] * FLOPS_BLEND) / 1e12
        return dict(kernel=dom, bound="alu", achieved=work / t, peak=alu_peak, unit="TFLOP/s",
                    frac=(work / t) / alu_peak, traffic=measured_traffic(dom),
                    note=f"{FLOPS_ALPHA} FP32 FLOPs per alpha test, over the whole tile list for pixels that "
                         f"cannot have saturated and up to n_last for the {100 * info['maybe_stopped']:.1f}% that "
                         f"may have (a lower bound), + {FLOPS_BLEND} per blend up to n_last, at the sampled SM clock")
    if dom == "render_backward":
        work = info["evals_per_step"] * FLOPS_BWD / 1e12
        return dict(kernel=dom, bound="alu", achieved=work / t, peak=alu_peak, unit="TFLOP/s",
                    frac=(work / t) / alu_peak, traffic=measured_traffic(dom),
                    note=f"{FLOPS_BWD} FP32 FLOPs per (pixel, splat) replayed up to n_last, at the sampled SM clock")
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    if dom == "hybrid_step":
        byts = info["touched"] * 59 * 4 * 7
    elif dom == "project_gaussians":
        byts = n * (44 + 48) + info["visible"] * 192
    elif dom == "project_backward":
        byts = n * 5 + info["visible"] * 48 + info["touched"] * 236 * 2
    elif dom == "project_backward_update":  # params, m, v read and written; no gradient
        byts = n * 5 + info["visible"] * 48 + info["touched"] * 236 * 6
    elif dom == "bin_tiles":
        byts = info["n_isect"] * 44
    elif dom == "select_tiles":
        byts = tr.H * tr.W * 4
    else:  # loss: target gather, rgb, gradient, error and age maps
        byts = tr.H * tr.W * 2 + info["P"] * 48
    ach = byts / t / 1e9
    return dict(kernel=dom, bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                traffic=measured_traffic(dom))


def replica_throughput(total_ms: float, steps: int, world: int, dist=None, device=None) -> float:
    """Whole-job iters/s of `world` independent replicas that each timed
    `steps` steps in total_ms: the slowest rank bounds the job (max over the
    ranks, an all-reduce when a process group is given)."""
    import torch
    tot = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    return world * steps / (tot.item() * 1e-3)


def error_stats_time(tr, info, flush, clocks, peaks, reps: int = 7) -> dict:
    """The error back-projection statistics of Sec. 3.8 (Eq. 12) over the
    step's sampled pixels, two ways: fused into the backward replay
    (render_backward_sampled_stats: the backward's time with the sums less
    its time without) and as the separate pass after the loss
    (error_stats_sampled).  Device ms per call (events on the launch stream,
    L2 flushed before each; median of reps)."""
    import torch
    from paper_2606_15924_gb300 import binding as B
    stats = torch.zeros(tr.n, 4, device=tr.params["means"].device)
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(reps):
            flush.fill_(1.0)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return sorted(ms)[len(ms) // 2]

    def separate():
        B.error_stats_sampled(tr.proj, tr.ranges, tr.vals, tr.active_tiles, tr.n_active, tr.n_select, tr.pix_off,
                              tr.pix_idx, tr.n_pix, tr.ccam, tr.n_last, tr.err_pix, stats, stream=stream)

    def plain():
        B.render_backward_sampled(tr.proj, tr.ranges, tr.vals, tr.active_tiles, tr.n_active, tr.n_select,
                                  tr.pix_off, tr.pix_idx, tr.n_pix, tr.ccam, tr.bg, tr.T_final, tr.n_last, tr.dL,
                                  tr.grad2d, ckpt=tr.ckpt, stream=stream)

    def fused():
        B.render_backward_sampled_stats(tr.proj, tr.ranges, tr.vals, tr.active_tiles, tr.n_active, tr.n_select,
                                        tr.pix_off, tr.pix_idx, tr.n_pix, tr.ccam, tr.bg, tr.T_final, tr.n_last,
                                        tr.dL, tr.grad2d, tr.err_pix, stats, ckpt=tr.ckpt, stream=stream)
    t_sep, t_plain, t_fused = timed(separate), timed(plain), timed(fused)
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    alu_peak = alu_peak_tflops(sm_mhz)
    achieved = info["evals_per_step"] * 27 / (t_sep * 1e-3) / 1e12
    return {"fused_backward_ms": t_fused, "plain_backward_ms": t_plain, "fused_extra_ms": t_fused - t_plain,
            "separate_pass_ms": t_sep, "separate_pass_roofline": {"bound": "alu", "achieved": achieved,
                                                                  "unit": "TFLOP/s", "frac": achieved / alu_peak},
            "note": "Sec. 3.8 statistics over the step's sampled pixels, fused into the backward replay or as the "
                    "separate walk; not in the timed step"}


VIEWS_V, VIEWS_K = 256, 10


def views_bench(device, peaks, flush, reps: int = 5) -> dict:
    """Geometry-aware view sampling (Sec. 3.4, Eqs. 5-6) over 256 views of
    1280 x 720 fp16 error maps: the per-view error totals (one pass over the
    472 MB of maps, HBM-bound; algorithmic bytes = V H W 2) and the draw of
    K = 10 views (one block).  Device ms per call, events on the launch
    stream, L2 flushed before each repetition."""
    import torch
    from paper_2606_15924_gb300 import scenes
    from paper_2606_15924_gb300.views import ViewSampler
    cams = scenes.orbit(VIEWS_V, DISTANCE, WIDTH, HEIGHT)
    gen = torch.Generator(device=device).manual_seed(11)
    maps = (torch.rand(VIEWS_V, HEIGHT, WIDTH, device=device, generator=gen) * 0.1).half().view(torch.int16)
    vs = ViewSampler(cams, seed=0)
    stream = torch.cuda.current_stream()
    for i in range(3):
        vs.error_sums(maps)
        vs.draw(VIEWS_K, i)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_sum, t_draw = [], []
    for i in range(reps):
        flush.fill_(1.0)
        ev[0].record(stream)
        vs.error_sums(maps)
        ev[1].record(stream)
        vs.draw(VIEWS_K, 3 + i)
        ev[2].record(stream)
        ev[2].synchronize()
        t_sum.append(ev[0].elapsed_time(ev[1]))
        t_draw.append(ev[1].elapsed_time(ev[2]))
    ts, td = sorted(t_sum)[reps // 2], sorted(t_draw)[reps // 2]
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = VIEWS_V * HEIGHT * WIDTH * 2 / (ts * 1e-3) / 1e9
    return {"views": VIEWS_V, "K": VIEWS_K, "maps": f"{VIEWS_V} x {WIDTH}x{HEIGHT} fp16", "error_sums_ms": ts,
            "draw_ms": td, "error_sums_roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                                                   "unit": "GB/s", "frac": achieved / hbm},
            "note": "Sec. 3.4 view draw of the multi-view step; not in the timed single-view step"}


def e2e_replays(tr, loss_host, steps):
    """Public-API step with the view's target copied in from pinned host memory
    and the loss read back, every step.  The trainer was captured with
    target_host and loss_host: each replayed step copies the target in itself,
    beside the kernels that do not read it (the loss waits for the copy), and
    its loss out to loss_host, beside the backward and update."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(4):  # warm-up: the first replays of these graphs also upload them
        tr.replay(with_copy=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(steps):
        tr.replay(with_copy=True)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    if not math.isfinite(float(loss_host[0])):
        raise RuntimeError("end-to-end steps read back a non-finite loss")
    return steps / (ms * 1e-3), tr.target.numel() * 4, loss_host.numel() * loss_host.element_size()


class OracleStep:
    """The oracle's sampled training step on a bounded sample of the
    workload, for the CPU baseline and the reference arm.

    Every run covers the whole selection, projection, projection adjoint and
    hybrid update of all Gaussians, and the render + loss + backward of the
    first ``k`` active tiles of the selection (whole tiles, so the loss has its
    tile statistics).  The target is the same second seeded Gaussian set the
    GPU arm renders, evaluated by the oracle at the sample's pixels (set-up,
    not timed); the error and age maps are seeded (the GPU arm's map comes
    from a dense render, which the oracle cannot afford per run).  ``run``
    returns the wall time of the sample and the modelled time of a full step
    (the tile part scaled to all of the step's sampled pixels)."""

    def __init__(self, cam, g_np, k_tiles=None, tile_budget_s=3.0):
        import numpy as np
        import oracle
        from paper_2606_15924_gb300 import scenes
        self.np, self.oracle, self.cam = np, oracle, cam
        T = ((WIDTH + 15) // 16) * ((HEIGHT + 15) // 16)
        self.n_sel = round(TILE_FRACTION * T)
        self.n_pix = math.floor(PIXEL_RATE * 256)
        self.err = scenes.error_map(WIDTH, HEIGHT)
        self.age = scenes.age_map(WIDTH, HEIGHT)
        self.g64 = {k: v.astype(np.float64) for k, v in g_np.items()}
        self.sel = oracle.select(self.err, self.age, WIDTH, HEIGHT, n_select=self.n_sel, n_pix=self.n_pix, seed=0)
        self.pix_all = oracle.pixel_coords(self.sel["active_tiles"], self.sel["pix_off"], self.sel["pix_idx"], WIDTH)
        self.P = len(self.pix_all)
        gt = scenes.gaussians(N_GAUSS, seed=scenes.SEED_TARGET, extent=EXTENT)
        self.pr_gt = oracle.project({k: v.astype(np.float64) for k, v in gt.items()}, cam)
        self.target = np.zeros((HEIGHT, WIDTH, 3))
        self.pk = np.concatenate([self.g64["means"], self.g64["log_scales"], self.g64["quats"],
                                  self.g64["opacity_logits"][:, None], self.g64["sh"].reshape(N_GAUSS, 48)], 1)
        if k_tiles is None:   # calibrate: whole tiles until the tile part takes about tile_budget_s
            k = 2
            while True:
                self.set_tiles(k)
                t0 = time.perf_counter()
                self._tiles(self.oracle.project(self.g64, cam, tile_rank=self.sel["tile_rank"]))
                if time.perf_counter() - t0 > tile_budget_s / 2 or k >= len(self.sel["active_tiles"]):
                    break
                k = min(len(self.sel["active_tiles"]), 2 * k)
            k_tiles = k
        self.set_tiles(k_tiles)

    def set_tiles(self, k):
        self.k = int(k)
        off = self.sel["pix_off"]
        self.sub = dict(active_tiles=self.sel["active_tiles"][:k], pix_off=off[:k + 1], pix_idx=self.sel["pix_idx"][:off[k]])
        self.pix = self.pix_all[:off[k]]
        t = self.oracle.render_pixels(self.pr_gt, WIDTH, HEIGHT, self.pix)["rgb"]
        self.target[self.pix[:, 1], self.pix[:, 0]] = t

    def _tiles(self, pr):
        r = self.oracle.render_pixels(pr, WIDTH, HEIGHT, self.pix)
        lo = self.oracle.loss(WIDTH, HEIGHT, self.sub, r["rgb"], self.target)
        return self.oracle.render_backward(pr, WIDTH, HEIGHT, self.pix, lo["dL_drgb"])

    def run(self):
        np, oracle = self.np, self.oracle
        t0 = time.perf_counter()
        sel = oracle.select(self.err, self.age, WIDTH, HEIGHT, n_select=self.n_sel, n_pix=self.n_pix, seed=0)
        pr = oracle.project(self.g64, self.cam, tile_rank=sel["tile_rank"])
        t1 = time.perf_counter()
        g2 = self._tiles(pr)
        t2 = time.perf_counter()
        grads = oracle.project_backward(self.g64, self.cam, g2, tile_rank=sel["tile_rank"])
        touched = (np.abs(g2).sum(1) > 0).astype(np.uint8)
        oracle.hybrid_step(self.pk, grads, np.zeros_like(self.pk), np.zeros_like(self.pk), touched, 1, 1,
                           [1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4, 0.9, 0.999, 1e-15, 1e-8])
        t3 = time.perf_counter()
        wall = t3 - t0
        modelled = (t1 - t0) + (t2 - t1) * (self.P / len(self.pix)) + (t3 - t2)
        return wall, modelled

    def describe(self):
        return (f"each run: selection, projection, projection adjoint and update of all {N_GAUSS} Gaussians, and "
                f"render+loss+backward of {len(self.pix)} of the step's {self.P} sampled pixels ({self.k} whole "
                f"tiles); the full step is modelled by scaling the tile part by {self.P / len(self.pix):.1f}; "
                f"target: the second seeded Gaussian set rendered by the oracle; seeded error/age maps")


def omp_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_baseline(cam, g_np, runs=2):
    """The oracle as it stands on a bounded sample of the same step (a few
    runs of OracleStep, about 10-30 s of CPU work in all)."""
    st = OracleStep(cam, g_np)
    res = [st.run() for _ in range(runs)]
    wall = sum(r[0] for r in res) / runs
    model = sum(r[1] for r in res) / runs
    return {"value": 1.0 / model, "unit": "iters/s", "cores": omp_threads(), "kind": "oracle", "modelled": True,
            "sample": st.describe() + f"; {runs} runs of {wall:.2f} s wall each, modelled step {model:.1f} s"}


def run_ours(args):
    import numpy as np
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2606_15924_gb300 import binding as B
    B.device_check()
    from paper_2606_15924_gb300.pipeline import psnr
    peaks, peak_kind = load_peaks()
    cam, g_np, target = build_scene(device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    sampled = make_trainer(g_np, cam, target, False, args.fraction, args.rate, device)
    dense = None if args.no_dense else make_trainer(g_np, cam, target, True, 1.0, 1.0, device)
    # each replay makes the next iteration's selection beside its own backward;
    # the end-to-end steps also copy the target in from pinned host memory,
    # beside the projection, binning and render, and copy the loss out beside
    # the backward
    tgt_host = target.detach().cpu().pin_memory()
    loss_host = torch.zeros(1, dtype=torch.float64, pin_memory=True)
    sampled.capture(overlap=True, target_host=tgt_host, loss_host=loss_host)
    if dense is not None:
        dense.capture(overlap=True)
    for _ in range(args.warmup):
        sampled.replay()
        if dense is not None:
            dense.replay()
    torch.cuda.synchronize()
    if args.profile:
        for name, tr in (("sampled_step", sampled), ("dense_step", dense)):
            if tr is None:
                continue
            torch.cuda.nvtx.range_push(name)
            for _ in range(args.steps):
                tr.replay()
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        return
    clk = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    t_wall = time.perf_counter()
    ms_s = time_replays(sampled, args.steps, flush)
    ms_d = time_replays(dense, args.steps, flush) if dense is not None else None
    t_wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    clocks = clk.stop()
    if dist is not None:
        dist.barrier()
    mean_s = sum(ms_s) / len(ms_s)
    value = replica_throughput(sum(ms_s), args.steps, world, dist, device)
    launches = sampled.kernels_per_step
    # per-stage times, roofline of the dominant kernel (eager pass, events on the launch stream)
    st, info = stage_times(sampled, max(2, min(args.steps, 5)), flush)
    roof = roofline(st, info, peaks, peak_kind, clocks, sampled)
    roof["peak_source"] = f"{peak_kind} (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback"
    stage_roofs = {k: roofline(st, info, peaks, peak_kind, clocks, sampled, dom=k) for k in st}
    fwdbwd_ms = st["render_sampled"] + st["render_backward"] + st.get("project_backward",
                                                                       st.get("project_backward_update", 0.0))
    mpix = info["P"] / (fwdbwd_ms * 1e-3) / 1e6
    err_stats = error_stats_time(sampled, info, flush, clocks, peaks)
    view_draw = views_bench(device, peaks, flush)
    res = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": mean_s, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded scenes; the paper's datasets are not "
                                                         "available)",
           "config": workload_config(args.fraction, args.rate), "gpu_launches": launches * args.steps,
           "roofline": roof, "clocks": clocks,
           "sampled": {"iters_per_s": 1e3 / mean_s, "ms_per_step": mean_s, "sampled_pixels": info["P"],
                       "active_tiles": info["A"], "tile_pairs": info["n_isect"], "touched": info["touched"],
                       "visible": info["visible"], "splat_evals": info["evals_per_step"],
                       "alpha_tests": info["walked_per_step"], "maybe_stopped": info["maybe_stopped"],
                       "tile_lists": info["tiles"],
                       "fwd_bwd_mpix_per_s": mpix, "stage_ms": st, "kernels_per_step": launches,
                       "error_stats": err_stats, "view_sampling": view_draw,
                       "stage_rooflines": {k: {"bound": v["bound"], "achieved": v["achieved"], "unit": v["unit"],
                                               "frac": v["frac"]} for k, v in stage_roofs.items()}}}
    if ms_d is not None:
        mean_d = sum(ms_d) / len(ms_d)
        st_d, info_d = stage_times(dense, 2, flush)
        res["dense"] = {"iters_per_s": 1e3 / mean_d, "ms_per_step": mean_d, "pixels": info_d["P"],
                        "fwd_bwd_mpix_per_s": info_d["P"] / ((st_d["render_sampled"] + st_d["render_backward"] +
                                                               st_d.get("project_backward",
                                                                        st_d.get("project_backward_update", 0.0)))
                                                              * 1e-3) / 1e6,
                        "stage_ms": st_d}
        res["speedup_vs_dense"] = mean_d / mean_s
    # end to end through the public API: target in from pinned host memory, loss out
    e2e_v, h2d, d2h = e2e_replays(sampled, loss_host, args.steps)
    res["e2e"] = {"value": e2e_v * world, "unit": "iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    res["mlp"] = mlp_bench(device, peaks)
    if not args.no_batched:
        del sampled, dense
        torch.cuda.empty_cache()
        sampled = dense = None
        res["batched"] = batched_summary(batched_measure(argparse.Namespace(rate=args.rate, warmup=3, steps=5,
                                                                            profile=False)))
        torch.cuda.empty_cache()
    if not args.no_quality:
        del sampled, dense
        torch.cuda.empty_cache()
        res["quality"] = quality_summary(held_out_quality(device, args))
    if rank == 0 and not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline(cam, g_np)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


# ---------------------------------------------------------------------------
# batched multi-view workload
# ---------------------------------------------------------------------------

N_BATCH_GAUSS = 3_000_000
BW, BH = 1920, 1080
N_BATCH_VIEWS = 8
N_ORBIT = 120


def batched_scene(device):
    """3M Gaussians; 8 views of a 120-view orbit at 1920x1080 with active-tile
    fractions drawn from U[3%, 60%]; targets = renders of a seeded
    ground-truth cloud plus N(0, 0.01) noise."""
    import numpy as np
    import torch
    from paper_2606_15924_gb300 import scenes
    from paper_2606_15924_gb300.pipeline import Trainer
    cams_all = scenes.orbit(N_ORBIT, DISTANCE, BW, BH)
    rng = np.random.default_rng(scenes.SEED_MASK)
    ids = sorted(int(i) for i in rng.choice(N_ORBIT, N_BATCH_VIEWS, replace=False))
    fracs = [float(f) for f in rng.uniform(0.03, 0.60, N_BATCH_VIEWS)]
    cams = [cams_all[i] for i in ids]
    gt = scenes.gaussians(N_BATCH_GAUSS, seed=scenes.SEED_TARGET, extent=EXTENT)
    gt_d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in gt.items()}
    gen = torch.Generator().manual_seed(scenes.SEED_NOISE)
    dummy = torch.zeros(BH, BW, 3, device=device)
    targets = []
    for cam in cams:
        img = Trainer(gt_d, cam, dummy, dense=True, train=False).render_image()
        noise = torch.randn(BH, BW, 3, generator=gen) * 0.01
        targets.append((img + noise.to(device)).contiguous())
    del gt_d
    torch.cuda.empty_cache()
    g = scenes.gaussians(N_BATCH_GAUSS, seed=scenes.SEED_SCENE, extent=EXTENT)
    from paper_2606_15924_gb300.pipeline import as_geo_rows
    params = as_geo_rows({k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in g.items()})
    return params, cams, targets, ids, fracs


def run_batched(args):
    """8 views per iteration in one persistent launch (forward and backward)
    against one launch per view, both inside a captured graph (one JSON
    line)."""
    print(json.dumps(batched_measure(args)))


def batched_summary(res: dict) -> dict:
    """The batched workload's figures for the headline line."""
    keep = ("iters_per_s", "ms_per_step", "views_per_step", "sampled_pixels", "render_fwd_ms", "render_bwd_ms",
            "fwd_bwd_mpix_per_s", "grid")
    out = {"workload": res["config"]["workload"], "speedup_vs_per_view": res["speedup_vs_per_view"]}
    for arm in ("persistent", "per_view"):
        a = res[arm]
        out[arm] = {k: a[k] for k in keep}
        out[arm]["render_fwd_roofline"] = a["render_fwd_roofline"]
        out[arm]["stage_ms"] = a["stage_ms"]
    return out


def batched_measure(args):
    import torch
    from paper_2606_15924_gb300 import binding as B
    from paper_2606_15924_gb300.batched import MultiViewTrainer, autotune_grid
    B.device_check()
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    peaks, peak_kind = load_peaks()
    params, cams, targets, ids, fracs = batched_scene(device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    out = {}
    for persistent in (True, False):
        mv = MultiViewTrainer(params, cams, targets, fracs, pixel_rate=args.rate, view_ids=ids,
                              persistent=persistent)
        for v in mv.views:
            v.init_error_map()
        mv.step()
        torch.cuda.synchronize()
        tune = autotune_grid(mv, reps=5, use_cache=False) if persistent else None
        mv.capture()
        for _ in range(args.warmup):
            mv.replay()
        torch.cuda.synchronize()
        if args.profile:  # replays inside an NVTX range for an ncu launch list, persistent launches only
            torch.cuda.nvtx.range_push("batched_step")
            for _ in range(args.steps):
                mv.replay()
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            return
        clk = ClockSampler(0)
        clk.start()
        ms = time_replays(mv, args.steps, flush)
        clocks = clk.stop()
        # every call of the step as its own graph, events between them
        st = stage_times_graphs(mv, max(2, min(args.steps, 5)), flush)
        fm, bm = st["render_sampled"], st["render_backward"]
        P = mv.n_sampled()
        evals = sum(int(v.n_last[:int(v.pix_off[int(v.n_active.item())].item())].sum().item())
                    for v in mv.views)
        mean = sum(ms) / len(ms)
        sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        alu_peak = alu_peak_tflops(sm_mhz)
        out["persistent" if persistent else "per_view"] = {
            "iters_per_s": 1e3 / mean, "ms_per_step": mean, "views_per_step": mv.K,
            "sampled_pixels": P, "active_tiles": [int(v.n_active.item()) for v in mv.views],
            "render_fwd_ms": fm, "render_bwd_ms": bm, "fwd_bwd_mpix_per_s": P / ((fm + bm) * 1e-3) / 1e6,
            "splat_evals": evals, "grid": list(mv.grid) if persistent else "one block per active tile",
            "stage_ms": st,
            "kernels_per_step": mv.kernels_per_step, "clocks": clocks,
            "render_fwd_roofline": {"bound": "alu", "achieved": evals * (FLOPS_ALPHA + FLOPS_BLEND) / (fm * 1e-3) / 1e12,
                                    "peak": alu_peak, "unit": "TFLOP/s"},
            "autotune": tune}
        out["persistent" if persistent else "per_view"]["render_fwd_roofline"]["frac"] = (
            out["persistent" if persistent else "per_view"]["render_fwd_roofline"]["achieved"] / alu_peak)
        del mv
        torch.cuda.empty_cache()
    res = {"metric": "batched multi-view train iters/s (8 views per iteration)",
           "value": out["persistent"]["iters_per_s"], "unit": "iters/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": out["persistent"]["ms_per_step"], "higher_is_better": True,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"batched views: {N_BATCH_GAUSS // 10**6}M Gaussians, {N_BATCH_VIEWS} views of a "
                                  f"{N_ORBIT}-view orbit at {BW}x{BH}, tile fractions U[3%,60%], "
                                  f"pixel rate {args.rate:.3f}", "views": ids, "tile_fractions": fracs,
                      "l2": "flushed between timed steps (256 MB write)"},
           "peak_source": peak_kind, **out,
           "speedup_vs_per_view": out["per_view"]["ms_per_step"] / out["persistent"]["ms_per_step"]}
    return res


MLP_ROWS = 200 * 8487   # tile rows of a 200-view orbit at 1957x1091


def mlp_bench(device, peaks, steps: int = 10, rows: int = MLP_ROWS) -> dict:
    """The tile-error MLP's forward and training step over one row per tile of
    a 200-view set, against the bf16 tensor peak: 2 (16*128 + 128*128 + 128)
    FLOPs per row forward, twice that more for the backward."""
    import torch
    from paper_2606_15924_gb300 import binding as B
    from paper_2606_15924_gb300.predictor import TileErrorMLP, HID
    R = int(rows)
    mlp = TileErrorMLP(device)
    g = torch.Generator(device="cpu").manual_seed(4)
    x = torch.randn(R, 16, generator=g).to(device)
    t = torch.randn(R, generator=g).to(device)
    y = torch.empty(R, device=device)
    h1 = torch.empty(R, HID, dtype=torch.int16, device=device)
    h2 = torch.empty(R, HID, dtype=torch.int16, device=device)
    ws = torch.empty(B.mlp_backward_workspace_size(R), dtype=torch.uint8, device=device)

    status = torch.zeros(1, dtype=torch.int32, device=device)

    def fwd():
        B.mlp_forward(mlp.net(), x, y, h1, h2)

    def fwd_tc():
        B.mlp_forward_tc(mlp.net(), x, y, h1, h2, status=status)

    def infer_tc():
        B.mlp_forward_tc(mlp.net(), x, y, status=status)

    def train():
        fwd()
        B.mlp_backward(mlp.net(), x, h1, h2, y, t, mlp.grads, mlp.loss, workspace=ws)
        B.mlp_adam(mlp.params, mlp.grads, mlp.m, mlp.v, 1, 1e-4, 0.9, 0.999, 1e-8, mlp.net())

    def train_tc():
        fwd_tc()
        B.mlp_backward_tc(mlp.net(), x, h1, h2, y, t, mlp.grads, mlp.loss, status=status, workspace=ws)
        B.mlp_adam(mlp.params, mlp.grads, mlp.m, mlp.v, 1, 1e-4, 0.9, 0.999, 1e-8, mlp.net())

    def train_fused():
        B.mlp_train_tc(mlp.net(), x, t, mlp.grads, mlp.loss, status=status)
        B.mlp_adam(mlp.params, mlp.grads, mlp.m, mlp.v, 1, 1e-4, 0.9, 0.999, 1e-8, mlp.net())

    def bwd():
        B.mlp_backward(mlp.net(), x, h1, h2, y, t, mlp.grads, mlp.loss, workspace=ws)

    def bwd_tc():
        B.mlp_backward_tc(mlp.net(), x, h1, h2, y, t, mlp.grads, mlp.loss, status=status, workspace=ws)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / steps
    f_ms, t_ms = timed(fwd), timed(train)
    ftc_ms, itc_ms = timed(fwd_tc), timed(infer_tc)
    b_ms, btc_ms, ttc_ms = timed(bwd), timed(bwd_tc), timed(train_tc)
    tfu_ms = timed(train_fused)
    flop = 2.0 * R * (16 * 128 + 128 * 128 + 128)
    peak = float(peaks.get("bf16_tflops", 1900.0))

    def roof(ms, note):
        a = flop / (ms * 1e-3) / 1e12
        return {"bound": "tensor", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak, "note": note}
    return {"rows": R, "forward_ms": f_ms, "forward_tc_ms": ftc_ms, "inference_tc_ms": itc_ms,
            "train_step_ms": t_ms, "tc_status": int(status.item()),
            "forward_roofline": roof(f_ms, "mma.sync m16n8k16 bf16, fp32 accumulate, h1/h2 stored"),
            "forward_tc_roofline": roof(ftc_ms, "tcgen05.mma bf16, TMEM accumulators, h1/h2 stored"),
            "inference_tc_roofline": roof(itc_ms, "tcgen05.mma bf16, TMEM accumulators, y only"),
            "peak_note": "peak = measured cuBLAS bf16 (burst)",
            "train_roofline": {"achieved": 3 * flop / (t_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                               "frac": 3 * flop / (t_ms * 1e-3) / 1e12 / peak},
            "backward_ms": b_ms, "backward_tc_ms": btc_ms, "train_step_tc_ms": ttc_ms,
            "train_tc_roofline": {"achieved": 3 * flop / (ttc_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                                  "frac": 3 * flop / (ttc_ms * 1e-3) / 1e12 / peak,
                                  "note": "tcgen05 forward with stored activations, tcgen05 activation "
                                          "adjoint, tcgen05 weight gradients, Adam"},
            "train_step_fused_ms": tfu_ms,
            "train_fused_roofline": {"achieved": 3 * flop / (tfu_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                                     "frac": 3 * flop / (tfu_ms * 1e-3) / 1e12 / peak,
                                     "note": "one tcgen05 kernel: forward recomputed, activation adjoint and "
                                             "weight gradients with the activations on chip; then Adam"}}


def run_quality(args):
    import torch
    from paper_2606_15924_gb300 import binding as B
    B.device_check()
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    res = held_out_quality(device, args)
    for v in res["sampled"].values():
        v.pop("curve", None)
    print(json.dumps({"metric": "sampled vs dense training at equal held-out PSNR (device time)", **res}))


QUALITY_VIEWS = 32


def held_out_quality(device, args):
    """Dense against sampled training at equal held-out PSNR: the bench's
    500k-Gaussian cloud on a 32-view orbit at 1280x720 with every eighth view
    held out, starting from the ground truth with every parameter jittered,
    targets with N(0, 0.01^2) noise; each sampled setting one view per step,
    and the paper's scheduled multi-view iteration (Sec. 3.4, App. A)."""
    from paper_2606_15924_gb300.quality import compare_views
    return compare_views(device, n=N_GAUSS, width=WIDTH, height=HEIGHT, distance=DISTANCE, extent=EXTENT,
                         n_views=QUALITY_VIEWS, dense_iters=args.dense_iters, settings=quality_settings(args),
                         scheduled=True, scheduled_fraction=args.fraction, mean_sigma=0.004, init="jitter")


def quality_settings(args):
    """The bench's own (tile fraction, pixel rate), the paper's sampling in
    every tile (a third and a tenth of the pixels), and half of the tiles at a
    tenth of their pixels (the best of the settings measured on this workload:
    20-100% of the tiles at 5-33% of their pixels all reach the dense held-out
    PSNR in 45-55% of the dense time)."""
    out = [(args.fraction, args.rate), (1.0, PIXEL_RATE), (1.0, 0.1), (0.5, 0.1)]
    return list(dict.fromkeys(out))


def quality_summary(res):
    """Compact per-setting result of a quality comparison for the bench line."""
    out = {"workload": res["workload"], "psnr": res.get("psnr", "trained view, every pixel"),
           "dense_psnr_db": res["dense"]["psnr"], "dense_iters": res["dense"]["iters"], "dense_ms": res["dense"]["ms"],
           "dense_iters_per_s": res["dense"]["iters_per_s"], "psnr_goal_db": res["psnr_goal"]}
    best = None
    for name, s in res["sampled"].items():
        out[name] = {k: s.get(k) for k in ("tile_fraction", "pixel_rate", "views_per_iter", "iters_per_s_ratio",
                                           "reached", "time_to_goal_ms", "dense_time_to_goal_ms", "time_speedup",
                                           "psnr", "iters", "ms")}
        if s.get("time_speedup") and (best is None or s["time_speedup"] > out[best]["time_speedup"]):
            best = name
    out["best_time_speedup"] = {"setting": best, "value": out[best]["time_speedup"] if best else None,
                                "target": 3.0}
    return out


def run_reference(args):
    """The oracle as the reference arm: rank 0 only, each step one bounded
    sample of the same workload on the host cores (OracleStep).  ``steps`` and
    ``ms_per_step`` are what ran (the samples' wall time); ``value`` is the
    modelled full-step rate, marked as modelled."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2606_15924_gb300 import scenes
    cam = scenes.look_at((0.0, 0.0, -DISTANCE), width=WIDTH, height=HEIGHT, fov_x_deg=60.0)
    g = scenes.gaussians(N_GAUSS, seed=scenes.SEED_SCENE, extent=EXTENT)
    # keep the whole run within a few minutes: about 150 s of timed and warm-up samples
    st = OracleStep(cam, g, tile_budget_s=max(0.5, 150.0 / max(1, args.steps + args.warmup) - 3.0))
    for _ in range(args.warmup):
        st.run()
    walls, models = [], []
    for _ in range(args.steps):
        w, m = st.run()
        walls.append(w)
        models.append(m)
    wall = sum(walls) / len(walls)
    v = len(models) / sum(models)
    cpu = {"value": v, "unit": "iters/s", "cores": omp_threads(), "kind": "oracle", "modelled": True,
           "sample": st.describe() + f"; {args.steps} timed runs of {wall:.2f} s wall each"}
    print(json.dumps({"metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": int(os.environ.get("WORLD_SIZE",
                                                                                                    "1")),
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall, "modelled": True,
                      "modelled_ms_per_full_step": 1e3 / v, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": workload_config(), "impl": "reference", "cpu_baseline": cpu,
                      "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fraction", type=float, default=TILE_FRACTION)
    ap.add_argument("--rate", type=float, default=PIXEL_RATE)
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--quality", action="store_true",
                    help="only the equal-quality comparison: dense training for a fixed number of iterations, then "
                         "sampled training until it is within 0.1 dB of the dense PSNR (device time)")
    ap.add_argument("--dense-iters", type=int, default=3000)
    ap.add_argument("--no-quality", action="store_true", help="skip the equal-PSNR comparison in the default run")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched multi-view workload's summary in the default run")
    ap.add_argument("--mlp-rows", type=int, default=0,
                    help="only the tile-error MLP kernels on this many rows (for a small profile), one JSON line")
    ap.add_argument("--workload", default="step", choices=["step", "batched"],
                    help="step: the one-view sparse training step (the headline line); batched: 8 views per "
                         "iteration in one persistent launch vs one launch per view")
    ap.add_argument("--profile", action="store_true",
                    help="only warm-up and K replays of each path inside NVTX ranges sampled_step / dense_step "
                         "(for an ncu launch list); prints nothing")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mlp_rows > 0:
        import torch
        from paper_2606_15924_gb300 import binding as B
        B.device_check()
        peaks, _ = load_peaks()
        print(json.dumps({"metric": "tile-error MLP", **mlp_bench(torch.device("cuda", 0), peaks,
                                                                 rows=args.mlp_rows)}))
    elif args.quality:
        run_quality(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

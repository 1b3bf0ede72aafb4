"""Several views per training iteration, rasterised in one persistent launch.

At iteration t the method trains on a set of K views (Alg. 1 steps 2-10; the
loss of Eq. 11 is an expectation over them).  ``MultiViewTrainer`` keeps one
``Trainer`` per view for the per-view state (error and age maps, sampled
tiles and pixels, projection, tile lists) and shares the Gaussians, their
gradients and the optimiser moments.  One step:

  per view: select_tiles -> project_gaussians -> bin_tiles
  all views: render_sampled_batched (one persistent launch, (view, tile) queue)
  per view: loss_sparse_ncc (view_weight 1/K)
  all views: render_backward_batched (one persistent launch)
  all views: project_backward_multi (one pass summing the views' adjoints
            into the shared gradients, and writing each view's Jacobian
            row for the Cholesky mode)
  once:     hybrid_step

Everything is sized at construction and the iteration counters live on the
device, so the step is captured once in a CUDA graph.  ``autotune_grid``
picks the persistent grid sizes by timing graph replays.

A trainer may also hold a pool of more views than it trains at once
(``max_active``): ``set_views`` then picks the views (and pixels per tile) of
the next steps, as the adaptive schedule and geometry-aware view sampling of
Sec. 3.4 do every iteration (``ScheduledTrainer``).  Every pool view keeps
its own maps and buffers resident; the active set's batch descriptors are
rebuilt on the host, and such steps run without a captured graph.
"""
from __future__ import annotations

import json
import os

import torch

from . import binding as B
from .config import Config
from .pipeline import Trainer, zeros_like_params


class MultiViewTrainer:
    def __init__(self, params: dict, cams: list, targets: list, tile_fractions: list,
                 pixel_rate: float = 1.0 / 3.0, cfg: Config | None = None, seed: int = 0, bg=(0.0, 0.0, 0.0),
                 sh_degree: int = 3, view_ids: list | None = None, grid: tuple | None = None,
                 view_rows: bool | None = None, persistent: bool = True, checkpoints: bool | None = None,
                 max_active: int | None = None, stats: bool = False):
        if not cams or len(cams) != len(targets) or len(cams) != len(tile_fractions):
            raise ValueError("one target and one tile fraction per view")
        # views trained together (one batch of the persistent launches)
        self.max_active = min(len(cams), 16) if max_active is None else int(max_active)
        if not 1 <= self.max_active <= 16 or (max_active is None and len(cams) > 16):
            raise ValueError("1 to 16 views per step (a larger pool needs max_active)")
        self.cfg = cfg or Config()
        self.params = params
        self.n = int(params["means"].shape[0])
        self.sh_degree, self.bg = sh_degree, tuple(bg)
        dev = params["means"].device
        ids = view_ids if view_ids is not None else list(range(len(cams)))
        self.pool = [Trainer(params, cams[k], targets[k], tile_fraction=tile_fractions[k], pixel_rate=pixel_rate,
                             cfg=self.cfg, seed=seed, bg=bg, sh_degree=sh_degree, view=ids[k], train=False)
                     for k in range(len(cams))]
        self.views = self.pool[:self.max_active]
        self.K = len(self.views)
        # one device iteration counter for all views (the hash of each view's
        # draw also takes its view id)
        self.it_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        self.step_dev = torch.ones(1, dtype=torch.int32, device=dev)
        w = 1.0 / self.K
        for v in self.pool:
            v.it_dev = self.it_dev
            v.loss_params = (v.loss_params[0], v.loss_params[1], v.loss_params[2], w)
            v.grad2d = torch.zeros(self.n, 12, device=dev)
        self.grads = zeros_like_params(params)
        self.m = zeros_like_params(params)
        self.v = zeros_like_params(params)
        self.touched = torch.zeros(self.n, dtype=torch.uint8, device=dev)
        # Eq. 12's statistics over the views' sampled pixels, accumulated step after step (persistent launch)
        if stats and not persistent:
            raise ValueError("the statistics ride on the persistent backward")
        self.stats = torch.zeros(self.n, 4, device=dev) if stats else None
        self.ws_hybrid = torch.empty(B.hybrid_step_workspace_size(self.n), dtype=torch.uint8, device=dev)
        self.ws_adj = torch.empty(B.project_backward_multi_workspace_size(self.n), dtype=torch.uint8, device=dev)
        o = self.cfg.opt
        self.opt = dict(lr=[o.lr_means, o.lr_scales, o.lr_quats, o.lr_opacity, o.lr_sh_dc, o.lr_sh_rest],
                        beta1=o.beta1, beta2=o.beta2, eps_adam=o.eps_adam, eps_lm=o.eps_lm, mode=o.mode)
        # per-view Jacobian rows feed only the full-matrix LM mode
        self.use_rows = (self.opt["mode"] == 2) if view_rows is None else bool(view_rows)
        self.rows = torch.zeros(self.max_active, self.n, 14, device=dev) if self.use_rows else None
        # persistent=False: one launch per view with one block per active
        # tile (the same kernels without the shared queue) and one
        # accumulating projection adjoint per view, for comparison
        self.persistent = bool(persistent)
        self.counters = torch.zeros(2 + 2 * self.max_active, dtype=torch.int32, device=dev)
        self.n_pix_max = max(v.n_pix for v in self.pool)
        # checkpoints for the split backward: one slot every CKPT_EVERY list
        # positions, up to CKPT_POSITIONS
        if checkpoints is None:
            # with the persistent launch the warp-per-piece backward beats the
            # whole-tile one even when the views' tiles fill the GPU (8 views
            # of 3M Gaussians at 1920x1080: 1.57 against 1.70 ms); one launch
            # per view keeps the whole-tile kernel (its pieces past the last
            # slot would run as one long tail per tile).  Checkpoints cost
            # n_pix x 64 float4 per active tile.
            checkpoints = self.persistent
        self.ck_slots = Trainer.CKPT_POSITIONS // Trainer.CKPT_EVERY if checkpoints else 0
        for v in self.pool:
            if self.ck_slots:
                v.ck_data = torch.empty(B.checkpoint_bytes(v.n_select, v.n_pix, self.ck_slots) // 4, device=dev)
                v.ck_last = torch.zeros(v.n_select, dtype=torch.int32, device=dev)
                v.ckpt = B.checkpoints(v.ck_data, self.ck_slots, v.n_select * v.n_pix, v.rgb, v.ck_last)
            else:
                v.ckpt = None
        res_f = B.render_batched_resident(self.n_pix_max, False)
        res_b = B.render_batched_resident(self.n_pix_max, 2 if self.ck_slots else 1)
        self.resident = (res_f, res_b)
        self.grid = tuple(grid) if grid is not None else (res_f, res_b)
        self._build_batches()
        self.graph = None

    def _build_batches(self):
        fwd, bwd = [], []
        for v in self.views:
            d = dict(proj=v.proj, tile_ranges=v.ranges, vals=v.vals, active_tiles=v.active_tiles,
                     n_active=v.n_active, n_active_max=v.n_select, pix_off=v.pix_off, pix_idx=v.pix_idx,
                     n_pix_max=v.n_pix, cam=v.ccam, bg=v.bg, rgb=v.rgb, T_final=v.T_final, n_last=v.n_last,
                     ckpt=v.ckpt)
            fwd.append(dict(d))
            d.update(dL_drgb=v.dL, grad2d=v.grad2d)
            bwd.append(d)
        # ctypes arrays hold raw pointers: rebuilt whenever a buffer is reallocated
        self.fwd_batch = B.view_batch(fwd)
        self.bwd_batch = B.view_batch(bwd)
        self.fwd_single = [B.view_batch([d]) for d in fwd]
        self.bwd_single = [B.view_batch([d]) for d in bwd]
        self.adj = B.MultiAdjoint([v.ccam for v in self.views], [v.proj["radius"] for v in self.views],
                                  [v.grad2d for v in self.views],
                                  [self.rows[k] for k in range(self.K)] if self.use_rows else None)

    def set_views(self, ids, n_pix: int | None = None):
        """Trains pool views ``ids`` (at most max_active, distinct) from the
        next step on, each with loss weight 1/len(ids) and, when given, n_pix
        sampled pixels per tile (at most the pixels the pool was sized for).
        Steps after this run eagerly (a captured graph holds the old set)."""
        ids = [int(i) for i in ids]
        if not 1 <= len(ids) <= self.max_active or len(set(ids)) != len(ids) or \
                not all(0 <= i < len(self.pool) for i in ids):
            raise ValueError("1 to max_active distinct pool views")
        views = [self.pool[i] for i in ids]
        if n_pix is not None and not all(1 <= n_pix <= v.P_max // v.n_select for v in views):
            raise ValueError("n_pix above the pool's allocation")
        self.views, self.K = views, len(views)
        w = 1.0 / self.K
        for v in views:
            v.loss_params = (v.loss_params[0], v.loss_params[1], v.loss_params[2], w)
            if n_pix is not None:
                v.n_pix = int(n_pix)
        self._build_batches()
        self.graph = None

    def _project_bwd(self):
        """Projection adjoint of all views into the shared gradients: one fused
        pass (persistent) or one accumulating launch per view."""
        if self.persistent:
            B.project_backward_multi(self.params, self.adj, self.grads, self.touched, write_untouched=False,
                                     sh_degree=self.sh_degree, workspace=self.ws_adj)
            return
        self.touched.zero_()
        for k, v in enumerate(self.views):
            B.project_backward(self.params, v.ccam, v.proj, v.grad2d, self.grads, self.touched,
                               write_untouched=False, accumulate=True,
                               view_row=self.rows[k] if self.use_rows else None, sh_degree=self.sh_degree)

    def _render_fwd(self):
        if self.persistent:
            B.render_sampled_batched(self.fwd_batch, self.grid[0], self.counters[0:1])
        else:
            for k, v in enumerate(self.views):
                B.render_sampled_batched(self.fwd_single[k], max(1, v.n_select), self.counters[2 + k:3 + k])

    def reset_stats(self):
        """Zeroes the accumulated statistics (after a density-control step)."""
        if self.stats is not None:
            self.stats.zero_()

    def _render_bwd(self):
        if self.persistent and self.stats is not None:
            B.render_backward_batched_stats(self.bwd_batch, self.grid[1], self.counters[1:2],
                                            [v.err_pix for v in self.views], self.stats, accumulate=True)
        elif self.persistent:
            B.render_backward_batched(self.bwd_batch, self.grid[1], self.counters[1:2])
        else:
            for k, v in enumerate(self.views):
                B.render_backward_batched(self.bwd_single[k], max(1, v.n_select * (self.ck_slots + 1)),
                                          self.counters[2 + self.K + k:3 + self.K + k])

    # ------------------------------------------------------------------ step
    def forward(self):
        for v in self.views:
            v._select()
            B.project_gaussians(self.params, v.ccam, v.tile_rank, v.proj, self.sh_degree)
            B.bin_tiles(v.proj, self.n, v.ccam, v.tile_rank, v.n_select, v.ws_bin, v.capacity, v.vals, None,
                        v.ranges, v.n_isect)
        self._render_fwd()

    def loss_and_maps(self):
        for v in self.views:
            v.loss_and_maps()

    def backward(self):
        self._render_bwd()
        self._project_bwd()

    def update(self):
        B.hybrid_step(self.params, self.grads, self.m, self.v, self.n, self.touched, self.rows,
                      self.K if self.use_rows else 0, 1, self.opt, workspace=self.ws_hybrid, step_dev=self.step_dev)

    @property
    def fused(self) -> bool:
        """Adjoint and update in one pass: the fused path of the persistent
        trainer in modes 0 and 1 (no per-view rows)."""
        return self.persistent and self.opt["mode"] in (0, 1) and not self.use_rows

    def backward_update(self):
        B.project_backward_update(self.params, self.adj, self.m, self.v, self.touched, self.opt, 1,
                                  step_dev=self.step_dev, sh_degree=self.sh_degree, workspace=self.ws_adj)

    def step(self):
        self.forward()
        self.loss_and_maps()
        if self.fused:
            self._render_bwd()
            self.backward_update()
        else:
            self.backward()
            self.update()
        B.advance_counters(self.it_dev, self.step_dev)

    def loss(self) -> float:
        """Mean loss over the views of the last step (reads the device)."""
        return float(sum(v.loss.item() for v in self.views))

    def overflowed(self) -> bool:
        return any(v.overflowed() for v in self.views)

    def n_sampled(self) -> int:
        """Sampled pixels of the last step over all views (reads the device)."""
        return int(sum(int(v.pix_off[int(v.n_active.item())].item()) for v in self.views))

    STAGES = ("select_tiles", "project_gaussians", "bin_tiles", "render_sampled", "loss_sparse_ncc",
              "render_backward", "project_backward", "hybrid_step")

    def stage_calls(self):
        """The step as (name, callable) pairs, each call over all views."""
        def select():
            for v in self.views:
                v._select()

        def project():
            for v in self.views:
                B.project_gaussians(self.params, v.ccam, v.tile_rank, v.proj, self.sh_degree)

        def bins():
            for v in self.views:
                B.bin_tiles(v.proj, self.n, v.ccam, v.tile_rank, v.n_select, v.ws_bin, v.capacity, v.vals, None,
                            v.ranges, v.n_isect)

        def upd():
            self.update()
            B.advance_counters(self.it_dev, self.step_dev)
        tail = ([("project_backward_update", lambda: (self.backward_update(),
                                                      B.advance_counters(self.it_dev, self.step_dev)))]
                if self.fused else [("project_backward", self._project_bwd), ("hybrid_step", upd)])
        return [("select_tiles", select), ("project_gaussians", project), ("bin_tiles", bins),
                ("render_sampled", self._render_fwd), ("loss_sparse_ncc", self.loss_and_maps),
                ("render_backward", self._render_bwd)] + tail

    def capture_stages(self):
        self.stage_graphs = []
        torch.cuda.synchronize()
        for name, fn in self.stage_calls():
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr):
                fn()
            self.stage_graphs.append((name, gr))
        torch.cuda.synchronize()
        return self.stage_graphs

    # ------------------------------------------------------------------ graph
    def capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph(keep_graph=True)
        with torch.cuda.graph(self.graph):
            self.step()
        self.kernels_per_step = B.graph_count_kernels(self.graph)
        self.graph.instantiate()
        torch.cuda.synchronize()
        return self.graph

    def replay(self):
        self.graph.replay()

    def capture_render(self):
        """Graphs of the two persistent launches alone (for timing and tuning)."""
        torch.cuda.synchronize()
        self.g_fwd = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.g_fwd):
            self._render_fwd()
        self.g_bwd = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.g_bwd):
            self._render_bwd()
        torch.cuda.synchronize()


# ---------------------------------------------------------------------- tuner
def _time_graph(g, reps: int) -> float:
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def grid_candidates(resident: int, sms: int) -> list:
    """Persistent grid sizes worth trying: whole waves of SMs up to the
    resident limit, plus the limit itself."""
    out = {resident}
    k = 1
    while k * sms < resident:
        out.add(k * sms)
        k *= 2
    return sorted(x for x in out if x >= 1)


def _cache_path() -> str:
    root = os.environ.get("TURBOGS_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "turbogs"))
    return os.path.join(root, "grid_tune.json")


def autotune_grid(mv: MultiViewTrainer, reps: int = 10, use_cache: bool = True) -> dict:
    """Pick (forward, backward) persistent grid sizes for this trainer's shape
    by timing graph replays of the two launches on the current sampled sets.
    The choice is cached per (device, views, image sizes, tile counts, pixels
    per tile) in a JSON file; returns {"grid": (f, b), "times": {...}}."""
    props = torch.cuda.get_device_properties(mv.params["means"].device)
    key = "|".join([props.name, str(mv.K)] + [f"{v.W}x{v.H}:{v.n_select}:{v.n_pix}" for v in mv.views])
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        mv.grid = tuple(cache[key]["grid"])
        return cache[key]
    sms = props.multi_processor_count
    times = {"fwd": {}, "bwd": {}}
    best = list(mv.grid)
    for which in (0, 1):
        best_t = None
        for g in grid_candidates(mv.resident[which], sms):
            grid = list(mv.grid)
            grid[which] = g
            mv.grid = tuple(grid)
            mv.capture_render()
            t = _time_graph(mv.g_fwd if which == 0 else mv.g_bwd, reps)
            times["fwd" if which == 0 else "bwd"][g] = t
            if best_t is None or t < best_t:
                best_t, best[which] = t, g
        grid = list(mv.grid)
        grid[which] = best[which]
        mv.grid = tuple(grid)
    result = {"grid": list(mv.grid), "times": times}
    if use_cache:
        cache[key] = result
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            json.dump(cache, open(path, "w"), indent=1)
        except OSError:
            pass
    return result

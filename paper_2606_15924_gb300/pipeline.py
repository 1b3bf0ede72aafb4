"""One TurboGS training iteration on the GPU, built from the C-ABI calls.

A ``Trainer`` owns the device buffers of one view's sparse step and runs,
in order (Alg. 1 steps 3-10): select_tiles -> project_gaussians -> bin_tiles ->
render_sampled -> loss_sparse_ncc (with the error/age map update) ->
backward_sampled -> hybrid_step; for the Adam and diagonal-LM modes the
projection adjoint and the update run as one call (project_backward_update),
and a sparse step keeps forward checkpoints for the warp-per-piece backward.
Sizes are fixed at construction and the
iteration counters live on the device, so one step can be captured once in a
CUDA graph and replayed.  ``dense=True`` gives the same library's plain path:
every tile active and every pixel sampled.
"""
from __future__ import annotations

import math

import torch

from . import binding as B
from .config import Config, TILE


def tiles_of(width: int, height: int) -> int:
    return ((width + TILE - 1) // TILE) * ((height + TILE - 1) // TILE)


_GEO = ("means", "log_scales", "quats", "opacity_logits")


def geo_stride_of(g: dict) -> int:
    """0 when the geometric fields are four packed arrays, else their row
    stride (views into one array of rows, ``binding.geo_rows``)."""
    return 0 if all(g[k].is_contiguous() for k in _GEO) else int(g["means"].stride(0))


def zeros_like_params(g: dict, n: int | None = None) -> dict:
    """Zero arrays shaped like the parameter set g (n rows, default g's), in
    the same layout of the geometric fields."""
    n = int(g["means"].shape[0]) if n is None else n
    dev, s = g["means"].device, geo_stride_of(g)
    if s:
        out = B.geo_rows(n, dev, s)
    else:
        out = {k: torch.zeros((n,) + tuple(g[k].shape[1:]), dtype=g[k].dtype, device=dev) for k in _GEO}
    out["sh"] = torch.zeros((n,) + tuple(g["sh"].shape[1:]), dtype=g["sh"].dtype, device=dev)
    return out


def as_geo_rows(g: dict, stride: int = 16) -> dict:
    """A copy of the parameter set g with its geometric fields in one array of
    rows of `stride` floats (64-byte rows at 16: an update of scattered
    Gaussians then moves whole rows instead of four partial sectors)."""
    n = int(g["means"].shape[0])
    out = B.geo_rows(n, g["means"].device, stride)
    for k in _GEO:
        out[k].copy_(g[k])
    out["sh"] = g["sh"].clone().contiguous()
    return out


def head_of(g: dict, m: int) -> dict:
    """The first m rows of g as a new parameter set of the same layout."""
    out = zeros_like_params(g, m)
    for k in out:
        out[k].copy_(g[k][:m])
    return out


class Trainer:
    CKPT_POSITIONS = 2048
    CKPT_EVERY = 32       # list positions per checkpoint slot (fixed by the kernels)

    def __init__(self, params: dict, cam: dict, target: torch.Tensor, tile_fraction: float = 0.2,
                 pixel_rate: float = 1.0 / 3.0, cfg: Config | None = None, dense: bool = False,
                 capacity: int | None = None, seed: int = 0, bg=(0.0, 0.0, 0.0), sh_degree: int = 3,
                 view: int = 0, train: bool = True, fuse_update: bool = True, share: "Trainer | None" = None,
                 stats: bool = False):
        """share: another view's trainer of the same Gaussians whose optimiser
        state (gradients, moments, step and iteration counters) this one uses,
        so that steps of several views' trainers form one training run.
        stats: the backward also accumulates the error back-projection
        statistics of Sec. 3.8 (Eq. 12) into self.stats [N,4] (E, W, D, 0),
        step after step until reset_stats()."""
        self.cfg = cfg or Config()
        self.fuse_update = fuse_update
        self.params = params
        self.n = int(params["means"].shape[0])
        self.cam = cam
        self.ccam = B.camera(cam)
        self.W, self.H = int(cam["width"]), int(cam["height"])
        self.T = tiles_of(self.W, self.H)
        self.dense = dense
        if dense:
            self.n_select, self.n_pix = self.T, 256
        else:
            self.n_select = max(1, min(self.T, round(tile_fraction * self.T)))
            self.n_pix = max(1, min(256, math.floor(pixel_rate * 256)))
        self.seed, self.view, self.bg, self.sh_degree = seed, view, tuple(bg), sh_degree
        self.target = target.contiguous()
        dev = params["means"].device
        i32, i64, u8 = torch.int32, torch.int64, torch.uint8
        T, N, S = self.T, self.n, self.n_select
        P = S * self.n_pix
        self.P_max = P
        # optimiser state (not needed for render-only use)
        self.train = train
        if train and share is not None:
            self.grads, self.m, self.v = share.grads, share.m, share.v
        elif train:
            self.grads = zeros_like_params(params)
            self.m = zeros_like_params(params)
            self.v = zeros_like_params(params)
        # per-view maps: fp16 error (bit patterns) and uint16 age
        self.err_map = torch.zeros(self.H, self.W, dtype=torch.int16, device=dev)
        self.age_map = torch.zeros(self.H, self.W, dtype=torch.int16, device=dev)
        # selection
        self.ws_sel = torch.empty(B.select_tiles_workspace_size(self.W, self.H), dtype=u8, device=dev)
        self.active_tiles = torch.zeros(S, dtype=i32, device=dev)
        self.n_active = torch.zeros(1, dtype=i32, device=dev)
        self.tile_rank = torch.zeros(T, dtype=i32, device=dev)
        self.pix_off = torch.zeros(S + 1, dtype=i32, device=dev)
        self.pix_idx = torch.zeros(P, dtype=u8, device=dev)
        # projection
        self.proj = dict(xy=torch.zeros(N, 2, device=dev), conic_opac=torch.zeros(N, 4, device=dev),
                         rgb=torch.zeros(N, 3, device=dev), depth=torch.zeros(N, device=dev),
                         radius=torch.zeros(N, dtype=i32, device=dev))
        # binning
        self.n_isect = torch.zeros(1, dtype=i64, device=dev)
        self.ranges = torch.zeros(S, 2, dtype=i32, device=dev)
        self.capacity = 0
        self._alloc_bins(capacity if capacity is not None else self._probe_capacity())
        # forward / loss / backward buffers
        self.rgb = torch.zeros(P, 3, device=dev)
        self.T_final = torch.zeros(P, device=dev)
        self.n_last = torch.zeros(P, dtype=i32, device=dev)
        self.dL = torch.zeros(P, 3, device=dev)
        self.lam = torch.zeros(S, device=dev)
        self.err_pix = torch.zeros(P, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        # forward checkpoints for the split backward: only when the step has
        # too few tiles to fill the GPU (sparse sampling); one slot every
        # CKPT_EVERY positions of the tile list up to CKPT_POSITIONS
        self.ckpt = None
        if train and not dense and self.n_select < 4 * B.render_batched_resident(self.n_pix, 1):
            n_slots = self.CKPT_POSITIONS // self.CKPT_EVERY
            self.ck_data = torch.empty(B.checkpoint_bytes(S, self.n_pix, n_slots) // 4, device=dev)
            self.ck_last = torch.zeros(S, dtype=torch.int32, device=dev)
            self.ckpt = B.checkpoints(self.ck_data, n_slots, S * self.n_pix, self.rgb, self.ck_last)
        self.stats = torch.zeros(N, 4, device=dev) if (train and stats) else None
        # the screen-space gradient statistic of the densification candidates (|dL/dxy| sum, count)
        self.accum = torch.zeros(N, 2, device=dev) if (train and stats) else None
        if train:
            self.grad2d = torch.zeros(N, 12, device=dev)
            self.touched = torch.zeros(N, dtype=u8, device=dev)
            self.ws_hybrid = torch.empty(B.hybrid_step_workspace_size(N), dtype=u8, device=dev)
            # the projection adjoint runs over a compacted list of the touched
            # Gaussians (the multi-view adjoint with one view)
            self.ws_adj = torch.empty(B.project_backward_multi_workspace_size(N), dtype=u8, device=dev)
            self.adj = B.MultiAdjoint([self.ccam], [self.proj["radius"]], [self.grad2d])
        # device-side counters (graph replays read them)
        if share is not None:
            self.it_dev, self.step_dev = share.it_dev, share.step_dev
        else:
            self.it_dev = torch.zeros(1, dtype=i64, device=dev)
            self.step_dev = torch.ones(1, dtype=i32, device=dev)
        self.graph = None
        o = self.cfg.opt
        self.opt = dict(lr=[o.lr_means, o.lr_scales, o.lr_quats, o.lr_opacity, o.lr_sh_dc, o.lr_sh_rest],
                        beta1=o.beta1, beta2=o.beta2, eps_adam=o.eps_adam, eps_lm=o.eps_lm, mode=o.mode)
        l = self.cfg.loss
        self.loss_params = (l.eps_charbonnier, l.eps_ncc, l.beta_ema)

    # ------------------------------------------------------------------ setup
    def _alloc_bins(self, capacity: int):
        dev = self.params["means"].device
        self.capacity = int(capacity)
        self.ws_bin = torch.empty(B.bin_tiles_workspace_size(self.n, self.capacity, self.n_select),
                                  dtype=torch.uint8, device=dev)
        self.vals = torch.zeros(max(self.capacity, 1), dtype=torch.int32, device=dev)

    def _probe_capacity(self) -> int:
        """Exact pair count of the dense view (one synchronising query at set-up),
        with headroom for the Gaussians moving during training."""
        dev = self.params["means"].device
        proj = dict(xy=torch.zeros(self.n, 2, device=dev), conic_opac=torch.zeros(self.n, 4, device=dev),
                    rgb=torch.zeros(self.n, 3, device=dev), depth=torch.zeros(self.n, device=dev),
                    radius=torch.zeros(self.n, dtype=torch.int32, device=dev))
        B.project_gaussians(self.params, self.ccam, None, proj, self.sh_degree)
        ws = torch.empty(B.bin_tiles_workspace_size(self.n, 0, self.T), dtype=torch.uint8, device=dev)
        ranges = torch.zeros(self.T, 2, dtype=torch.int32, device=dev)
        n_isect = torch.zeros(1, dtype=torch.int64, device=dev)
        B.bin_tiles(proj, self.n, self.ccam, None, self.T, ws, 0, None, None, ranges, n_isect)
        need = int(n_isect.item())
        return int(need * 1.3) + 4096

    def overflowed(self) -> bool:
        """True when the last step produced more tile pairs than the capacity
        (reads one device value; call outside the timed loop)."""
        return int(self.n_isect.item()) > self.capacity

    # ------------------------------------------------------------------ step
    def _select(self, n_select=None, n_pix=None, it_dev=True):
        B.select_tiles(self.err_map, self.age_map, self.W, self.H, n_select or self.n_select, n_pix or self.n_pix,
                       self.cfg.sampling.permille(), self.seed, 0, self.view, self.ws_sel, self.active_tiles,
                       self.n_active, self.tile_rank, self.pix_off, self.pix_idx,
                       iter_dev=self.it_dev if it_dev else None)

    def forward(self):
        """select -> project -> bin -> render (Alg. 1 steps 3, 5)."""
        self._select()
        B.project_gaussians(self.params, self.ccam, self.tile_rank, self.proj, self.sh_degree)
        B.bin_tiles(self.proj, self.n, self.ccam, self.tile_rank, self.n_select, self.ws_bin, self.capacity,
                    self.vals, None, self.ranges, self.n_isect)
        B.render_sampled(self.proj, self.ranges, self.vals, self.active_tiles, self.n_active, self.n_select,
                         self.pix_off, self.pix_idx, self.n_pix, self.ccam, self.bg, self.rgb, self.T_final,
                         self.n_last, ckpt=self.ckpt)

    def loss_and_maps(self):
        """Fused loss with the error/age map update (Alg. 1 steps 4, 6, 7)."""
        B.loss_sparse_ncc(self.rgb, self.target, self.W, self.H, self.active_tiles, self.n_active, self.n_select,
                          self.pix_off, self.pix_idx, self.n_pix, self.loss_params, self.err_map, self.age_map,
                          self.dL, self.lam, self.err_pix, self.loss, structure=self.cfg.loss.structure)

    def reset_stats(self):
        """Zeroes the accumulated statistics (after a density-control step)."""
        if self.stats is not None:
            self.stats.zero_()
            self.accum.zero_()

    def render_backward(self):
        """Compositing adjoint into grad2d (first half of Alg. 1 step 8); with
        stats, Eq. 12's sums of the same pixels in the same replay (Alg. 1
        step 11's back-projection)."""
        if self.stats is not None:
            B.render_backward_sampled_stats(self.proj, self.ranges, self.vals, self.active_tiles, self.n_active,
                                            self.n_select, self.pix_off, self.pix_idx, self.n_pix, self.ccam,
                                            self.bg, self.T_final, self.n_last, self.dL, self.grad2d, self.err_pix,
                                            self.stats, accumulate=True, ckpt=self.ckpt)
            B.accumulate_screen_grad(self.grad2d, self.accum)
            return
        B.render_backward_sampled(self.proj, self.ranges, self.vals, self.active_tiles, self.n_active,
                                  self.n_select, self.pix_off, self.pix_idx, self.n_pix, self.ccam, self.bg,
                                  self.T_final, self.n_last, self.dL, self.grad2d, ckpt=self.ckpt)

    def project_backward(self, write_untouched=False):
        """Projection adjoint into the parameter gradients (second half)."""
        B.project_backward_multi(self.params, self.adj, self.grads, self.touched, write_untouched=write_untouched,
                                 sh_degree=self.sh_degree, workspace=self.ws_adj)

    def backward(self, write_untouched=False):
        """Sparse backward into parameter gradients (Alg. 1 step 8)."""
        self.render_backward()
        self.project_backward(write_untouched)

    def update(self):
        """Hybrid LM / Adam update (Alg. 1 steps 9, 10)."""
        B.hybrid_step(self.params, self.grads, self.m, self.v, self.n, self.touched, None, 0, 1, self.opt,
                      workspace=self.ws_hybrid, step_dev=self.step_dev)

    def backward_update(self):
        """Projection adjoint and hybrid update in one pass (modes 0, 1):
        the parameter gradients are not written."""
        B.project_backward_update(self.params, self.adj, self.m, self.v, self.touched, self.opt, 1,
                                  step_dev=self.step_dev, sh_degree=self.sh_degree, workspace=self.ws_adj)

    @property
    def fused(self) -> bool:
        return self.fuse_update and self.opt["mode"] in (0, 1)

    def step(self):
        """One full iteration; advances the device counters."""
        self.forward()
        self.loss_and_maps()
        if self.fused:
            self.render_backward()
            self.backward_update()
        else:
            self.backward()
            self.update()
        B.advance_counters(self.it_dev, self.step_dev)

    # ------------------------------------------------------------------ graph
    SELECTION = ("ws_sel", "active_tiles", "n_active", "tile_rank", "pix_off", "pix_idx")

    def _selection(self) -> dict:
        return {k: getattr(self, k) for k in self.SELECTION}

    def _use_selection(self, sel: dict):
        for k, v in sel.items():
            setattr(self, k, v)

    def step_overlapped(self, nxt: dict, target_host=None, loss_host=None):
        """One iteration on the selection already made for it, and the next
        iteration's selection (Alg. 1 step 3) into the buffers nxt.  The next
        selection needs only the error and age maps the loss has just written
        and the iteration counter, so it runs on a second stream beside the
        backward and the update, which touch neither.  target_host (pinned
        host memory): the view's target is first copied in on a third stream,
        beside the projection, binning and render, which do not read it; the
        loss waits for it.  loss_host (pinned host memory, one float64): the
        loss is copied out on that stream too, beside the backward and update."""
        main = torch.cuda.current_stream()
        if target_host is not None:
            self._copy.wait_stream(main)
            with torch.cuda.stream(self._copy):
                self.target.copy_(target_host, non_blocking=True)
        B.project_gaussians(self.params, self.ccam, self.tile_rank, self.proj, self.sh_degree)
        B.bin_tiles(self.proj, self.n, self.ccam, self.tile_rank, self.n_select, self.ws_bin, self.capacity,
                    self.vals, None, self.ranges, self.n_isect)
        B.render_sampled(self.proj, self.ranges, self.vals, self.active_tiles, self.n_active, self.n_select,
                         self.pix_off, self.pix_idx, self.n_pix, self.ccam, self.bg, self.rgb, self.T_final,
                         self.n_last, ckpt=self.ckpt)
        if target_host is not None:
            main.wait_stream(self._copy)
        self.loss_and_maps()
        if loss_host is not None:
            self._copy.wait_stream(main)
            with torch.cuda.stream(self._copy):
                loss_host.copy_(self.loss, non_blocking=True)
        self._side.wait_stream(main)
        cur = self._selection()
        with torch.cuda.stream(self._side):
            # the next iteration's number, then its selection: off the main
            # stream, whose backward and update do not read the counter
            B.advance_counters(self.it_dev, None)
            self._use_selection(nxt)
            self._select()
        self._use_selection(cur)
        if self.fused:
            self.render_backward()
            self.backward_update()
        else:
            self.backward()
            self.update()
        B.advance_counters(None, self.step_dev)
        main.wait_stream(self._side)
        if loss_host is not None:
            main.wait_stream(self._copy)

    def capture(self, overlap: bool = False, target_host=None, loss_host=None):
        """Capture one step in a CUDA graph (after a warm-up step).  With
        overlap, two graphs that alternate between two sets of selection
        buffers: each runs its iteration on one set and makes the next
        iteration's selection in the other, beside its backward and update
        (``step_overlapped``); ``replay`` alternates them.  The results are
        those of the plain step: the same selections, from the same maps and
        counters.  With overlap and target_host (a pinned host copy of the
        target), a second pair of graphs whose steps also copy the target in
        from the host (``replay(with_copy=True)``); with loss_host too (pinned,
        one float64), those steps also copy their loss out to it, so that a
        replay leaves its loss in host memory once the device is done with it."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.overlap = overlap
        if not overlap:
            self.graph = torch.cuda.CUDAGraph(keep_graph=True)
            with torch.cuda.graph(self.graph):
                self.step()
            self.kernels_per_step = B.graph_count_kernels(self.graph)
            self.graph.instantiate()
            torch.cuda.synchronize()
            return self.graph
        self._side = torch.cuda.Stream()
        self._copy = torch.cuda.Stream()
        sets = [self._selection(), {k: torch.empty_like(v) for k, v in self._selection().items()}]
        self._select()                                  # the first replayed iteration's selection, in set 0
        torch.cuda.synchronize()

        def pair(host, out_host):
            out = []
            for k in range(2):
                self._use_selection(sets[k])
                g = torch.cuda.CUDAGraph(keep_graph=True)
                with torch.cuda.graph(g):
                    self.step_overlapped(sets[1 - k], host, out_host)
                out.append(g)
            return out
        self.graphs = pair(None, None)
        self.graphs_copy = pair(target_host, loss_host) if target_host is not None else None
        self.kernels_per_step = B.graph_count_kernels(self.graphs[0])
        for g in self.graphs + (self.graphs_copy or []):
            g.instantiate()
        self._sets, self._phase = sets, 0
        self._use_selection(sets[0])
        self.graph = self.graphs[0]
        torch.cuda.synchronize()
        return self.graph

    def replay(self, with_copy: bool = False):
        """One captured iteration.  With overlap, the selection attributes
        then name the buffers that iteration used (its rgb, n_last, ... go with
        them), and the next selection is already in the other set.  with_copy:
        the iteration that first copies the target in from the host (captured
        with target_host)."""
        if not getattr(self, "overlap", False):
            self.graph.replay()
            return
        k = self._phase
        self._use_selection(self._sets[k])
        (self.graphs_copy if with_copy else self.graphs)[k].replay()
        self._phase = 1 - k

    def next_selection(self) -> dict:
        """With overlap: the selection buffers of the next replayed iteration."""
        return self._sets[self._phase]

    STAGES = ("select_tiles", "project_gaussians", "bin_tiles", "render_sampled", "loss_sparse_ncc",
              "render_backward", "project_backward", "hybrid_step")

    def stage_calls(self):
        """The step as (name, callable) pairs, one per C-ABI call."""
        def bump():
            B.advance_counters(self.it_dev, self.step_dev)
        return [("select_tiles", self._select),
                ("project_gaussians", lambda: B.project_gaussians(self.params, self.ccam, self.tile_rank, self.proj,
                                                                  self.sh_degree)),
                ("bin_tiles", lambda: B.bin_tiles(self.proj, self.n, self.ccam, self.tile_rank, self.n_select,
                                                  self.ws_bin, self.capacity, self.vals, None, self.ranges,
                                                  self.n_isect)),
                ("render_sampled", lambda: B.render_sampled(self.proj, self.ranges, self.vals, self.active_tiles,
                                                            self.n_active, self.n_select, self.pix_off,
                                                            self.pix_idx, self.n_pix, self.ccam, self.bg, self.rgb,
                                                            self.T_final, self.n_last, ckpt=self.ckpt)),
                ("loss_sparse_ncc", self.loss_and_maps),
                ("render_backward", self.render_backward)] + (
                [("project_backward_update", lambda: (self.backward_update(), bump()))] if self.fused else
                [("project_backward", self.project_backward), ("hybrid_step", lambda: (self.update(), bump()))])

    def capture_stages(self):
        """One CUDA graph per call of the step, so each call's device time can
        be measured with events between replays (run after capture())."""
        self.stage_graphs = []
        torch.cuda.synchronize()
        for name, fn in self.stage_calls():
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr):
                fn()
            self.stage_graphs.append((name, gr))
        torch.cuda.synchronize()
        return self.stage_graphs

    # ------------------------------------------------------------------ maps
    def init_error_map(self, on_dense=None, want_loss: bool = True):
        """E_v from a dense evaluation of the current Gaussians (Sec. 3.3):
        every tile and pixel rendered once, E = e, A = 0.  Returns the loss
        (None without want_loss: nothing waits for the device).  on_dense(d)
        (optional) sees the dense evaluation after its loss.  The dense
        evaluator of a sampled trainer is kept for later refreshes."""
        if self.dense:
            d = self
        else:
            d = getattr(self, "_dense_eval", None)
            if d is None or d.n != self.n or d.params["means"].data_ptr() != self.params["means"].data_ptr():
                d = Trainer(self.params, self.cam, self.target, cfg=self.cfg, dense=True, seed=self.seed,
                            bg=self.bg, sh_degree=self.sh_degree, view=self.view, train=False)
                self._dense_eval = d
        d.err_map, d.age_map = self.err_map, self.age_map
        d.forward()
        saved = d.loss_params
        d.loss_params = (saved[0], saved[1], 1.0)
        d.loss_and_maps()
        d.loss_params = saved
        if on_dense is not None:
            on_dense(d)
        self.age_map.zero_()
        return float(d.loss.item()) if want_loss else None

    def render_image(self) -> torch.Tensor:
        """Dense render of the current Gaussians as an [H, W, 3] image (for
        evaluation; uses the same library calls)."""
        d = Trainer(self.params, self.cam, self.target, cfg=self.cfg, dense=True, seed=self.seed, bg=self.bg,
                    sh_degree=self.sh_degree, view=self.view, train=False)
        d.forward()
        return d.scatter_image(d.rgb)

    def pixel_coords(self):
        """[P, 2] integer pixel coordinates of the current sampled set (tile order)."""
        A = int(self.n_active.item())
        off = self.pix_off[:A + 1].long()
        counts = off[1:] - off[:-1]
        tiles = torch.repeat_interleave(self.active_tiles[:A].long(), counts)
        l = self.pix_idx[:int(off[-1])].long()
        tx_n = (self.W + TILE - 1) // TILE
        x = (tiles % tx_n) * TILE + (l % TILE)
        y = (tiles // tx_n) * TILE + (l // TILE)
        return torch.stack([x, y], 1)

    def scatter_image(self, per_pixel: torch.Tensor) -> torch.Tensor:
        xy = self.pixel_coords()
        img = torch.zeros(self.H, self.W, per_pixel.shape[-1], device=per_pixel.device, dtype=per_pixel.dtype)
        img[xy[:, 1], xy[:, 0]] = per_pixel[:xy.shape[0]]
        return img


def density_step(tr: Trainer, t: int, extent: float, final: bool = False) -> tuple[dict, dict, dict, int]:
    """One step of error-driven density control (Sec. 3.8, Eq. 13; Alg. 1
    step 11) on the statistics tr accumulated (Trainer(stats=True)) since its
    last reset, with the settings of tr.cfg.density: returns the new
    parameters, first and second moments (device tensors of the new count)
    and the count.  The caller builds the trainer of the new Gaussians and
    resets the statistics."""
    d = tr.cfg.density
    if tr.stats is None:
        raise ValueError("the trainer accumulates no statistics (stats=True)")
    rho = min(1.0, max(0.0, t / d.tau_until))
    cfg = B.density_params(d.lambda_base * (1.0 - rho), d.tau_grad, math.log(d.percent_dense * extent),
                           math.log(d.prune_opacity / (1.0 - d.prune_opacity)), topk_permille=round(1000 * d.topk),
                           final=final, final_permille=round(1000 * d.final_keep), eps=d.eps)
    cap = 2 * tr.n
    dev = tr.params["means"].device

    po, mo, vo = (zeros_like_params(x, cap) for x in (tr.params, tr.m, tr.v))
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    B.density_control(tr.params, tr.m, tr.v, tr.stats, tr.accum, cfg, po, mo, vo, cap, n_out,
                      sh_degree=tr.sh_degree)
    m = int(n_out.item())   # at most 2 N by construction
    return head_of(po, m), head_of(mo, m), head_of(vo, m), m


def psnr(img: torch.Tensor, ref: torch.Tensor) -> float:
    mse = torch.mean((img.clamp(0, 1) - ref) ** 2).item()
    return float(10.0 * math.log10(1.0 / max(mse, 1e-12)))

"""Learned tile-error predictor (an extension; the paper has no counterpart).

A 3-layer MLP (16 -> 128 -> 128 -> 1, ReLU; bf16 weights, fp32 accumulate)
run by the library's own kernels (forward on the tcgen05 tensor cores) predicts log(1 + mean tile error) from
per-tile features, so tile selection can use fresh predictions for views
whose error maps are stale instead of a dense refresh render.  Master weights
are fp32 (packed W1 | b1 | W2 | b2 | W3 | b3); the kernels read bf16 copies.
"""
from __future__ import annotations

import math

import torch

from . import binding as B

IN, HID = 16, 128


class TileErrorMLP:
    def __init__(self, device="cuda", seed: int = 0, lr: float = 1e-3):
        g = torch.Generator().manual_seed(seed)
        n = B.mlp_param_count()
        p = torch.zeros(n)          # biases start at zero
        sl = self._slices()
        for name, fan_in in (("W1", IN), ("W2", HID), ("W3", HID)):
            k = sl[name].stop - sl[name].start
            bound = math.sqrt(6.0 / fan_in)          # He-uniform for ReLU layers
            p[sl[name]] = (torch.rand(k, generator=g) * 2 - 1) * bound
        self.params = p.to(device)
        self.m = torch.zeros(n, device=device)
        self.v = torch.zeros(n, device=device)
        self.grads = torch.zeros(n, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.step_count = 0
        self.lr = lr
        self.w1 = torch.zeros(HID * IN, dtype=torch.int16, device=device)
        self.w2 = torch.zeros(HID * HID, dtype=torch.int16, device=device)
        self.w3 = torch.zeros(HID, dtype=torch.int16, device=device)
        self._refresh_bf16()

    # views into the packed master vector
    def _slices(self):
        o1 = HID * IN
        o2 = o1 + HID
        o3 = o2 + HID * HID
        o4 = o3 + HID
        o5 = o4 + HID
        return dict(W1=slice(0, o1), b1=slice(o1, o2), W2=slice(o2, o3), b2=slice(o3, o4), W3=slice(o4, o5),
                    b3=slice(o5, o5 + 1))

    def _refresh_bf16(self):
        sl = self._slices()
        for name, dst in (("W1", self.w1), ("W2", self.w2), ("W3", self.w3)):
            dst.copy_(self.params[sl[name]].to(torch.bfloat16).view(torch.int16))

    def net(self) -> dict:
        sl = self._slices()
        return dict(w1=self.w1, w2=self.w2, w3=self.w3, b1=self.params[sl["b1"]], b2=self.params[sl["b2"]],
                    b3=self.params[sl["b3"]])

    def weights_fp(self) -> dict:
        """Master weights as float64 numpy arrays (for checks)."""
        sl = self._slices()
        p = self.params.double().cpu().numpy()
        return dict(W1=p[sl["W1"]].reshape(HID, IN), b1=p[sl["b1"]], W2=p[sl["W2"]].reshape(HID, HID),
                    b2=p[sl["b2"]], W3=p[sl["W3"]], b3=p[sl["b3"]])

    def predict(self, x: torch.Tensor) -> torch.Tensor:
        """Inference on the tcgen05 tensor cores."""
        y = torch.empty(x.shape[0], device=x.device)
        B.mlp_forward_tc(self.net(), x.contiguous(), y)
        return y

    def train_step(self, x: torch.Tensor, target: torch.Tensor, rows_dev=None) -> torch.Tensor:
        """One Adam step on mean (y - t)^2 / 2 over the first rows_dev rows (all
        when None); returns the loss of the batch before the step (device)."""
        # forward and gradient in one tensor-core pass (no stored activations)
        B.mlp_train_tc(self.net(), x.contiguous(), target.contiguous(), self.grads, self.loss, rows_dev=rows_dev)
        self.step_count += 1
        B.mlp_adam(self.params, self.grads, self.m, self.v, self.step_count, self.lr, 0.9, 0.999, 1e-8, self.net())
        return self.loss


class TileMemory:
    """What one view last observed in each of its tiles (list length, mean
    final transmittance, mean error, iteration), kept on the device."""

    def __init__(self, n_tiles: int, device):
        self.mem = torch.zeros(n_tiles, 4, device=device)
        self.it = torch.zeros(n_tiles, dtype=torch.int64, device=device)


class TileErrorPredictor:
    """Online-trained tile-error predictor for a set of views.

    After each step's loss, ``observe_and_train`` forms the features of the
    step's active tiles from the view's tile memory as it was, records the new
    observations and takes one training step.  The network predicts a tile's
    log(1 + mean error) now; with residual=True it predicts instead the change
    since the tile's last observation, added to that stale value.  ``refresh`` brings a stale
    view's error map up to date before its next selection: with the network's
    predictions when its recent error (the loss of each batch before it was
    trained on, smoothed) is below ``max_mse``, otherwise with the plain
    refresh - a dense render of the view (Sec. 3.3), which is also what scores
    the network (``assess``)."""

    def __init__(self, device="cuda", seed: int = 0, lr: float = 1e-3, max_mse: float = 0.02,
                 min_batches: int = 50, residual: bool = False, replay: int = 2048, score_every: int = 1):
        self.mlp = TileErrorMLP(device, seed, lr)
        self.residual = residual
        self.device = device
        self.memories = {}
        self.max_mse, self.min_batches = max_mse, min_batches
        self.batches = 0
        self.recent_mse = None
        self.refreshes = {"predicted": 0, "plain": 0}
        # the network's error on the step's rows (a host read, so a wait for
        # the device) is taken every score_every-th batch
        self.score_every = max(1, int(score_every))
        # replay ring of the latest observations (features as they were, target):
        # each training step runs on all of it, not only on the step's few tiles
        self.replay = int(replay)
        self.buf_x = torch.zeros(max(self.replay, 1), IN, device=device)
        self.buf_t = torch.zeros(max(self.replay, 1), device=device)
        self.buf_n = 0
        self.buf_head = 0

    def _push(self, x: torch.Tensor, t: torch.Tensor):
        cap = self.replay
        A = x.shape[0]
        if A > cap:
            x, t, A = x[A - cap:], t[A - cap:], cap
        i = self.buf_head
        k = min(A, cap - i)
        self.buf_x[i:i + k] = x[:k]
        self.buf_t[i:i + k] = t[:k]
        if k < A:
            self.buf_x[:A - k] = x[k:]
            self.buf_t[:A - k] = t[k:]
        self.buf_head = (i + A) % cap
        self.buf_n = min(self.buf_n + A, cap)

    def memory(self, tr) -> TileMemory:
        if tr.view not in self.memories:
            self.memories[tr.view] = TileMemory(tr.T, self.device)
        return self.memories[tr.view]

    def init_view(self, tr, it: int = 0, want_loss: bool = True):
        """The plain refresh of a view (dense evaluation), also filling its
        tile memory; returns the loss (None without want_loss)."""
        mem = self.memory(tr)
        return tr.init_error_map(on_dense=lambda d: B.tile_observe(
            d.active_tiles, d.n_active, d.n_select, d.pix_off, d.ranges, d.T_final, d.err_pix, mem.mem, mem.it,
            None, it=it), want_loss=want_loss)

    def observe_and_train(self, tr, it: int, view_cos: float = 1.0, train: bool = True):
        """The step's active tiles: features from the memory as it was, then the
        new observations recorded; with train, the error on them before
        training (smoothed into recent_mse) and one Adam step.  With a replay
        ring the step trains on the ring (this step's rows and the latest
        before them), else on this step's rows alone.  The sampled step selects
        exactly n_select tiles, so every row of the batch is an observation."""
        mem = self.memory(tr)
        A = tr.n_select
        x = torch.zeros(A, IN, device=self.device)
        target = torch.zeros(A, device=self.device)
        B.tile_features(mem.mem, mem.it, tr.ccam, x, rows=tr.active_tiles, n_rows=tr.n_active, n_rows_max=A,
                        view_cos=view_cos, it=it)
        B.tile_observe(tr.active_tiles, tr.n_active, A, tr.pix_off, tr.ranges, tr.T_final, tr.err_pix, mem.mem,
                       mem.it, target, it=it, residual=self.residual)
        if not train:
            return
        score = self.batches % self.score_every == 0
        if self.replay:
            mse = float(((self.mlp.predict(x) - target) ** 2).mean().item()) if score else None
            self._push(x, target)
            self.mlp.train_step(self.buf_x[:self.buf_n], self.buf_t[:self.buf_n])
        else:
            loss = self.mlp.train_step(x, target, rows_dev=tr.n_active)
            mse = 2.0 * float(loss.item()) if score else None
        self.batches += 1
        if mse is not None:
            self.recent_mse = mse if self.recent_mse is None else 0.9 * self.recent_mse + 0.1 * mse

    def features(self, tr, it: int, view_cos: float = 1.0) -> torch.Tensor:
        mem = self.memory(tr)
        x = torch.empty(tr.T, 16, device=self.device)
        B.tile_features(mem.mem, mem.it, tr.ccam, x, n_rows_max=tr.T, view_cos=view_cos, it=it)
        return x

    def predict(self, tr, it: int, view_cos: float = 1.0) -> torch.Tensor:
        """Predicted log(1 + mean error) of every tile of the view [T]."""
        x = self.features(tr, it, view_cos)
        r = self.mlp.predict(x)
        return r + x[:, 2] if self.residual else r

    def trusted(self) -> bool:
        return self.batches >= self.min_batches and self.recent_mse is not None and self.recent_mse <= self.max_mse

    def refresh(self, tr, it: int, view_cos: float = 1.0) -> str:
        if self.trusted():
            x = self.features(tr, it, view_cos)
            B.tile_refresh(self.mlp.predict(x), tr.err_map, tr.W, tr.H, base=x if self.residual else None)
            self.refreshes["predicted"] += 1
            return "predicted"
        self.init_view(tr, it, want_loss=False)
        self.refreshes["plain"] += 1
        return "plain"

    def assess(self, tr, it: int, view_cos: float = 1.0) -> dict:
        """Scores the predictions for a view against a dense evaluation (the
        plain refresh) without changing the view's state: mean squared error
        of log(1 + tile error), and the same for the view's current error map."""
        from .pipeline import Trainer
        pred = self.predict(tr, it, view_cos)
        d = Trainer(tr.params, tr.cam, tr.target, cfg=tr.cfg, dense=True, seed=tr.seed, bg=tr.bg,
                    sh_degree=tr.sh_degree, view=tr.view, train=False)
        d.forward()
        d.loss_and_maps()
        truth = torch.zeros(tr.T, device=self.device)
        A = int(d.n_active.item())
        off = d.pix_off[:A + 1].long()
        cnt = (off[1:] - off[:-1]).clamp(min=1).float()
        seg = torch.repeat_interleave(torch.arange(A, device=self.device), off[1:] - off[:-1])
        truth.index_add_(0, d.active_tiles[:A].long()[seg], d.err_pix[:int(off[-1])])
        truth[d.active_tiles[:A].long()] /= cnt
        lt = torch.log1p(truth)
        stale = tile_means(tr.err_map, tr.W, tr.H)
        return dict(mse_pred=float(((pred - lt) ** 2).mean().item()),
                    mse_stale=float(((torch.log1p(stale) - lt) ** 2).mean().item()),
                    truth=lt, pred=pred, stale=torch.log1p(stale))


def tile_means(err_map: torch.Tensor, W: int, H: int) -> torch.Tensor:
    """Per-tile mean of an fp16 error map (bit patterns in int16), [T]."""
    from .config import TILE
    e = err_map.view(torch.float16).float()
    ty, tx = (H + TILE - 1) // TILE, (W + TILE - 1) // TILE
    pad = torch.zeros(ty * TILE, tx * TILE, device=e.device)
    ones = torch.zeros_like(pad)
    pad[:H, :W] = e
    ones[:H, :W] = 1.0
    s = pad.view(ty, TILE, tx, TILE).sum((1, 3))
    c = ones.view(ty, TILE, tx, TILE).sum((1, 3))
    return (s / c).reshape(-1)

"""Several views in one persistent launch: the batched forward renders every
(view, tile) item exactly as the one-view call renders it (bit-identical, for
any grid size), the batched backward gives the one-view compositing adjoint
(up to the order of float atomics), the accumulating projection adjoint sums
the views' gradients, the per-view Jacobian rows match each view's own
gradient, and the whole multi-view step runs from one captured CUDA graph."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu

W, H = 256, 192
FRACTIONS = [0.05, 0.3, 0.6, 0.2]


@pytest.fixture(scope="module")
def B():
    from paper_2606_15924_gb300 import binding
    binding.device_check()
    return binding


def _make(view_rows=False, mode=1, n=20000, checkpoints=None):
    from gpu_util import dev, gaussians_dev
    from paper_2606_15924_gb300.batched import MultiViewTrainer
    from paper_2606_15924_gb300.config import Config
    g = gaussians_dev(scenes.gaussians(n, seed=0))
    cams = scenes.orbit(3, 4.0, W, H)
    # a fourth view looking away from the scene: nothing visible
    cams.append(scenes.look_at((0.0, 0.0, -4.0), target=(0.0, 0.0, -10.0), width=W, height=H))
    targets = [dev(scenes.smooth_image(W, H, seed=10 + k)) for k in range(4)]
    cfg = Config()
    cfg.opt.mode = mode
    mv = MultiViewTrainer(g, cams, targets, FRACTIONS, cfg=cfg, view_rows=view_rows, checkpoints=checkpoints)
    for k, v in enumerate(mv.views):
        v.err_map.copy_(dev(scenes.error_map(W, H, seed=k).view(np.int16)))
    return mv


def _P(v):
    return int(v.pix_off[int(v.n_active.item())].item())


def _render_one(B, v):
    rgb, T, nl = torch.zeros_like(v.rgb), torch.zeros_like(v.T_final), torch.zeros_like(v.n_last)
    B.render_sampled(v.proj, v.ranges, v.vals, v.active_tiles, v.n_active, v.n_select, v.pix_off, v.pix_idx,
                     v.n_pix, v.ccam, v.bg, rgb, T, nl)
    return rgb, T, nl


def test_batched_forward_equals_per_view_bitwise(B):
    mv = _make()
    mv.forward()
    torch.cuda.synchronize()
    assert [v.n_select for v in mv.views] != [mv.views[0].n_select] * 4   # uneven tile counts
    for k, v in enumerate(mv.views):
        rgb, T, nl = _render_one(B, v)
        P = _P(v)
        assert P > 0
        assert torch.equal(rgb[:P], v.rgb[:P]), k
        assert torch.equal(T[:P], v.T_final[:P]), k
        assert torch.equal(nl[:P], v.n_last[:P]), k
    # the view looking away sees nothing: background everywhere, T = 1
    v = mv.views[3]
    assert int(v.n_isect.item()) == 0
    assert torch.all(v.rgb[:_P(v)] == 0) and torch.all(v.T_final[:_P(v)] == 1)
    assert int(mv.views[2].n_isect.item()) > 0


def test_batched_forward_independent_of_grid(B):
    mv = _make()
    mv.forward()
    torch.cuda.synchronize()
    ref = [v.rgb.clone() for v in mv.views]
    refT = [v.T_final.clone() for v in mv.views]
    for grid in (1, 7, 152, mv.resident[0]):
        for v in mv.views:
            v.rgb.zero_()
            v.T_final.zero_()
        B.render_sampled_batched(mv.fwd_batch, grid, mv.counters[0:1])
        torch.cuda.synchronize()
        for k, v in enumerate(mv.views):
            P = _P(v)
            assert torch.equal(v.rgb[:P], ref[k][:P]), (grid, k)
            assert torch.equal(v.T_final[:P], refT[k][:P]), (grid, k)


def _close(a, b, rel=2e-5):
    scale = float(b.abs().max().item()) if b.numel() else 0.0
    return float((a - b).abs().max().item()) <= rel * scale + 1e-9


@pytest.mark.parametrize("split", [False, True])
def test_batched_backward_and_accumulated_gradients(B, split):
    mv = _make(view_rows=True, mode=2, checkpoints=split)
    assert (mv.ck_slots > 0) == split
    mv.forward()
    mv.loss_and_maps()
    mv.backward()
    torch.cuda.synchronize()
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    total = {k: torch.zeros_like(mv.params[k]) for k in keys}
    union = torch.zeros(mv.n, dtype=torch.bool, device="cuda")
    for k, v in enumerate(mv.views):
        g2 = torch.zeros_like(v.grad2d)
        grads = {kk: torch.zeros_like(mv.params[kk]) for kk in keys}
        touched = torch.zeros(mv.n, dtype=torch.uint8, device="cuda")
        B.backward_sampled(mv.params, v.ccam, v.proj, v.ranges, v.vals, v.active_tiles, v.n_active, v.n_select,
                           v.pix_off, v.pix_idx, v.n_pix, v.bg, v.T_final, v.n_last, v.dL, g2, grads, touched,
                           write_untouched=True)
        torch.cuda.synchronize()
        assert _close(v.grad2d, g2), k
        for kk in keys:
            total[kk] += grads[kk]
        union |= touched.bool()
        # this view's Jacobian row (hybrid_step layout)
        row = torch.cat([grads["means"], grads["log_scales"], grads["quats"], grads["sh"][:, 0, :],
                         grads["opacity_logits"][:, None]], 1)
        assert _close(mv.rows[k], row), k
        if k == 3:
            assert not touched.any() and torch.all(mv.rows[k] == 0)
    assert torch.equal(mv.touched.bool(), union)
    assert int(union.sum().item()) > 100
    for kk in keys:
        assert _close(mv.grads[kk][union], total[kk][union]), kk


def test_view_weight_scales_loss_gradient_exactly(B):
    mv = _make()
    mv.forward()
    # maps untouched by the extra evaluation: pass no error/age map
    v = mv.views[1]
    lp = v.loss_params
    dL1 = torch.zeros_like(v.dL)
    lam, ep = torch.zeros_like(v.lam), torch.zeros_like(v.err_pix)
    loss1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.loss_sparse_ncc(v.rgb, v.target, v.W, v.H, v.active_tiles, v.n_active, v.n_select, v.pix_off, v.pix_idx,
                      v.n_pix, (lp[0], lp[1], lp[2], 1.0), None, None, dL1, lam, ep, loss1)
    B.loss_sparse_ncc(v.rgb, v.target, v.W, v.H, v.active_tiles, v.n_active, v.n_select, v.pix_off, v.pix_idx,
                      v.n_pix, lp, None, None, v.dL, v.lam, v.err_pix, v.loss)
    torch.cuda.synchronize()
    assert lp[3] == 0.25
    P = _P(v)
    assert torch.equal(v.dL[:P], dL1[:P] * 0.25)
    assert abs(v.loss.item() - 0.25 * loss1.item()) <= 1e-12 * abs(loss1.item())


def _dense_loss(dense):
    tot = 0.0
    for d in dense:
        d.forward()
        d.loss_and_maps()
        tot += d.loss.item()
    return tot


@pytest.mark.parametrize("mode,rows", [(1, False), (2, True)])
def test_multiview_step_in_one_graph_trains(B, mode, rows):
    from paper_2606_15924_gb300.pipeline import Trainer
    mv = _make(view_rows=rows, mode=mode)
    dense = [Trainer(mv.params, v.cam, v.target, dense=True, train=False) for v in mv.views[:3]]
    before = _dense_loss(dense)
    mv.capture()
    assert mv.kernels_per_step > 0
    for _ in range(40):
        mv.replay()
    torch.cuda.synchronize()
    after = _dense_loss(dense)
    assert np.isfinite(before) and np.isfinite(after)
    assert after < before
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        assert torch.isfinite(mv.params[k]).all()
    assert int(mv.it_dev.item()) == 41   # the eager warm-up step + 40 replays
    assert int(mv.step_dev.item()) == 42


def test_autotune_picks_a_candidate_and_keeps_results(B, tmp_path, monkeypatch):
    from paper_2606_15924_gb300.batched import autotune_grid, grid_candidates
    monkeypatch.setenv("TURBOGS_CACHE", str(tmp_path))
    mv = _make()
    mv.forward()
    torch.cuda.synchronize()
    ref = [v.rgb.clone() for v in mv.views]
    res = autotune_grid(mv, reps=2)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert mv.grid[0] in grid_candidates(mv.resident[0], sms)
    assert mv.grid[1] in grid_candidates(mv.resident[1], sms)
    assert (tmp_path / "grid_tune.json").exists()
    mv.grid = (1, 1)
    assert autotune_grid(mv)["grid"] == res["grid"]    # from the cache
    B.render_sampled_batched(mv.fwd_batch, mv.grid[0], mv.counters[0:1])
    torch.cuda.synchronize()
    for k, v in enumerate(mv.views):
        P = _P(v)
        assert torch.equal(v.rgb[:P], ref[k][:P])


def test_batched_rejects_bad_arguments(B):
    mv = _make(n=2000)
    with pytest.raises(B.TgsError):
        B.render_sampled_batched(mv.fwd_batch, 0, mv.counters[0:1])
    with pytest.raises(B.TgsError):
        B.render_sampled_batched(mv.fwd_batch, 152, None)
    with pytest.raises(B.TgsError):
        B.render_backward_batched(mv.fwd_batch, 152, mv.counters[1:2])   # no dL / grad2d


def test_fused_multiview_adjoint_equals_per_view_sum(B):
    mv = _make(view_rows=True, mode=2)
    mv.forward()
    mv.loss_and_maps()
    mv._render_bwd()
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    mv.persistent = True
    for k in keys:
        mv.grads[k].fill_(7.0)        # untouched entries are left alone
    mv._project_bwd()
    torch.cuda.synchronize()
    fused = {k: mv.grads[k].clone() for k in keys}
    fused_t = mv.touched.clone()
    fused_rows = mv.rows.clone()
    mv.persistent = False
    mv.rows.fill_(3.0)
    mv._project_bwd()
    torch.cuda.synchronize()
    assert torch.equal(fused_t, mv.touched)
    t = fused_t.bool()
    assert int(t.sum().item()) > 100
    for k in keys:
        assert _close(fused[k][t], mv.grads[k][t], rel=1e-5), k
        assert torch.all(fused[k][~t] == 7.0), k
    assert _close(fused_rows, mv.rows, rel=1e-6)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("views", [1, 4])
def test_fused_adjoint_update_equals_separate_calls(B, mode, views):
    """project_backward_update == project_backward_multi + hybrid_step on the
    same state (parameters, moments, touched), one view or several."""
    mv = _make(mode=mode)
    mv.forward()
    mv.loss_and_maps()
    mv._render_bwd()
    torch.cuda.synchronize()
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    rng = torch.Generator(device="cuda").manual_seed(5)
    m0 = {k: torch.rand(mv.m[k].shape, generator=rng, device="cuda") * 1e-3 for k in keys}
    v0 = {k: torch.rand(mv.v[k].shape, generator=rng, device="cuda") * 1e-4 for k in keys}
    p0 = {k: mv.params[k].clone() for k in keys}
    adj = mv.adj if views == 4 else B.MultiAdjoint([mv.views[1].ccam], [mv.views[1].proj["radius"]],
                                                   [mv.views[1].grad2d])
    step = torch.full((1,), 3, dtype=torch.int32, device="cuda")
    # separate calls
    pa = {k: p0[k].clone() for k in keys}
    ma = {k: m0[k].clone() for k in keys}
    va = {k: v0[k].clone() for k in keys}
    grads = {k: torch.zeros_like(p0[k]) for k in keys}
    ta = torch.zeros(mv.n, dtype=torch.uint8, device="cuda")
    B.project_backward_multi(pa, adj, grads, ta, write_untouched=False)
    B.hybrid_step(pa, grads, ma, va, mv.n, ta, None, 0, 1, mv.opt, step_dev=step)
    # fused
    pb = {k: p0[k].clone() for k in keys}
    mb = {k: m0[k].clone() for k in keys}
    vb = {k: v0[k].clone() for k in keys}
    tb = torch.zeros(mv.n, dtype=torch.uint8, device="cuda")
    B.project_backward_update(pb, adj, mb, vb, tb, mv.opt, 1, step_dev=step)
    torch.cuda.synchronize()
    assert torch.equal(ta, tb) and int(ta.sum().item()) > 100
    for k in keys:
        for a, b, name in ((pa[k], pb[k], "param"), (ma[k], mb[k], "m"), (va[k], vb[k], "v")):
            assert torch.allclose(a, b, rtol=1e-5, atol=1e-9), (k, name, float((a - b).abs().max()))
        untouched = ~ta.bool()
        assert torch.equal(pb[k][untouched], p0[k][untouched])     # untouched Gaussians keep their state

"""The batched multi-view step against the oracle (Alg. 1 steps 5-10 over the
views of one iteration; Eq. 11's expectation over views read as their mean).

Four views of a seeded 20k-Gaussian cloud (three on an orbit, one looking
away from the scene) with uneven tile fractions run through the persistent
launches the batched trainer uses: the forward over all (view, tile) items,
the fused loss per view with weight 1/K, the warp-per-piece backward from the
forward's checkpoints, and the fused projection adjoint of all views with
the hybrid update (diagonal LM, mode 1).  The oracle runs the same chain
view by view on its own: selection, projection, per-pixel render, loss,
compositing adjoint, projection adjoint summed over the views, one hybrid
step on the sum; and the error back-projection statistics of Sec. 3.8
(Eq. 12) that the batched backward accumulates over the views' pixels.
Every oracle input is the scene, the maps and the seeds; nothing comes from
the CUDA path."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu

W, H = 256, 192
FRACTIONS = [0.05, 0.3, 0.6, 0.2]
N = 20000
MARGIN = 1e-4


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _scene():
    g = scenes.gaussians(N, seed=0)
    cams = scenes.orbit(3, 4.0, W, H)
    cams.append(scenes.look_at((0.0, 0.0, -4.0), target=(0.0, 0.0, -10.0), width=W, height=H))
    targets = [scenes.smooth_image(W, H, seed=10 + k) for k in range(4)]
    errs = [scenes.error_map(W, H, seed=k) for k in range(4)]
    ages = [scenes.age_map(W, H, seed=40 + k) for k in range(4)]
    return g, cams, targets, errs, ages


def _pack(g):
    n = g["means"].shape[0]
    return np.concatenate([g["means"], g["log_scales"], g["quats"], g["opacity_logits"][:, None],
                           np.asarray(g["sh"]).reshape(n, 48)], 1).astype(np.float64)


def test_batched_step_against_oracle(orc):
    from paper_2606_15924_gb300 import binding as B
    from paper_2606_15924_gb300.batched import MultiViewTrainer
    from paper_2606_15924_gb300.config import Config
    from gpu_util import dev, gaussians_dev
    B.device_check()
    g, cams, targets, errs, ages = _scene()
    cfg = Config()
    cfg.opt.mode = 1
    params = gaussians_dev(g)
    mv = MultiViewTrainer(params, cams, [dev(t) for t in targets], FRACTIONS, cfg=cfg, seed=3)
    assert mv.persistent and mv.ck_slots > 0 and mv.fused
    for k, v in enumerate(mv.views):
        v.err_map.copy_(dev(errs[k].view(np.int16)))
        v.age_map.copy_(dev(ages[k].view(np.int16)))
    K = mv.K
    # moments of a step already under way (seeded), so the update is not a first step
    rng = np.random.default_rng(17)
    p0 = _pack(g)
    m0 = rng.normal(0.0, 1e-4, p0.shape)
    v0 = rng.uniform(1e-8, 1e-6, p0.shape)

    def split(a, like):
        t = torch.from_numpy(np.ascontiguousarray(a.astype(np.float32))).cuda()
        like["means"].copy_(t[:, 0:3])
        like["log_scales"].copy_(t[:, 3:6])
        like["quats"].copy_(t[:, 6:10])
        like["opacity_logits"].copy_(t[:, 10])
        like["sh"].copy_(t[:, 11:59].reshape(N, 16, 3))

    def join(d):
        return np.concatenate([d["means"].cpu().numpy(), d["log_scales"].cpu().numpy(), d["quats"].cpu().numpy(),
                               d["opacity_logits"].cpu().numpy()[:, None], d["sh"].cpu().numpy().reshape(N, 48)],
                              1).astype(np.float64)
    split(m0, mv.m)
    split(v0, mv.v)

    # --- the GPU: one multi-view iteration, phase by phase, as step() runs it
    mv.forward()
    mv.loss_and_maps()
    # the backward with Eq. 12's statistics of every view's sampled pixels (Sec. 3.8)
    stats = torch.zeros(N, 4, device="cuda")
    B.render_backward_batched_stats(mv.bwd_batch, mv.grid[1], mv.counters[1:2], [v.err_pix for v in mv.views],
                                    stats)
    step = 1
    B.project_backward_update(mv.params, mv.adj, mv.m, mv.v, mv.touched, mv.opt, step, step_dev=mv.step_dev)
    torch.cuda.synchronize()

    # --- the oracle, view by view
    g64 = {k: np.asarray(v, np.float64) for k, v in g.items()}
    grad_sum = np.zeros((N, 59))
    stats_o = np.zeros((N, 3))
    touched_o = np.zeros(N, bool)
    sure_g = np.ones(N, bool)
    n_pix_checked = 0
    for k, v in enumerate(mv.views):
        sel_o = orc.select(errs[k], ages[k], W, H, n_select=v.n_select, n_pix=v.n_pix, seed=3, it=0, view=k)
        A = int(v.n_active.item())
        assert A == sel_o["n_active"]
        np.testing.assert_array_equal(v.active_tiles[:A].cpu().numpy(), sel_o["active_tiles"])
        P = int(sel_o["pix_off"][-1])
        np.testing.assert_array_equal(v.pix_idx[:P].cpu().numpy(), sel_o["pix_idx"])
        prw = orc.project(g64, cams[k], tile_rank=sel_o["tile_rank"])
        sure_g &= prw["margin"] > MARGIN
        pix = orc.pixel_coords(sel_o["active_tiles"], sel_o["pix_off"], sel_o["pix_idx"], W)
        ro = orc.render_pixels(prw, W, H, pix)
        sure_p = ro["margin"] > MARGIN
        assert P > 0 and sure_p.mean() > 0.95
        # the batched forward at every sampled pixel of the view
        np.testing.assert_array_equal(v.n_last[:P].cpu().numpy()[sure_p], ro["n_last"][sure_p])
        assert np.abs(v.rgb[:P].cpu().numpy()[sure_p] - ro["rgb"][sure_p]).max() <= 1e-4
        assert np.abs(v.T_final[:P].cpu().numpy()[sure_p] - ro["T"][sure_p]).max() <= 1e-4
        n_pix_checked += int(sure_p.sum())
        # the view's loss on the oracle's own render, weighted 1/K (Eq. 11 over views)
        lo = orc.loss(W, H, sel_o, ro["rgb"], targets[k].astype(np.float64), err_f16_bits=errs[k], age=ages[k])
        assert float(v.loss.item()) == pytest.approx(lo["loss"] / K, rel=1e-4)
        dL_o = lo["dL_drgb"] / K
        assert rel_l2(v.dL[:P].cpu().numpy(), dL_o) <= 1e-3
        np.testing.assert_array_equal(v.age_map.cpu().numpy().view(np.uint16), lo["age_map"])
        # the view's compositing adjoint (warp-per-piece, persistent launch)
        g2o = orc.render_backward(prw, W, H, pix, dL_o)
        g2g = v.grad2d.cpu().numpy()
        if np.abs(g2o).sum() > 0:
            for c in range(9):
                assert rel_l2(g2g[sure_g, c], g2o[sure_g, c]) <= 1e-3, (k, c)
        else:
            assert k == 3 and not np.any(g2g)          # the view looking away sees nothing
        grad_sum += orc.project_backward(g64, cams[k], g2o, tile_rank=sel_o["tile_rank"])
        stats_o += orc.error_stats(prw, W, H, pix, lo["err"])
        touched_o |= (np.abs(g2o).sum(1) > 0) & (prw["radius"] > 0)
    assert n_pix_checked > 3000
    st_g = stats.cpu().numpy().astype(np.float64)
    assert (stats_o[sure_g, 1] > 0).sum() > 500
    for c in range(3):
        assert rel_l2(st_g[sure_g, c], stats_o[sure_g, c]) <= 1e-3, c

    # the fused adjoint of all views + one hybrid step on the summed gradient
    cfgv = np.array(mv.opt["lr"] + [mv.opt["beta1"], mv.opt["beta2"], mv.opt["eps_adam"], mv.opt["eps_lm"]])
    pw, mw, vw = orc.hybrid_step(p0, grad_sum, m0, v0, touched_o.astype(np.uint8), step, 1, cfgv)
    t_g = mv.touched.cpu().numpy().astype(bool)
    assert (t_g[sure_g] == touched_o[sure_g]).mean() > 0.999
    both = t_g & touched_o & sure_g
    assert both.sum() > 500
    pg = join(mv.params)
    p32 = p0.astype(np.float32).astype(np.float64)
    dp_g, dp_w = pg - p32, pw - p0
    ulp = np.spacing(np.abs(pw).astype(np.float32)).astype(np.float64)
    # parameters are stored in fp32: each element within its rounding plus the gradient tolerance
    within = np.abs(pg - pw) <= 1.5 * ulp + 2e-3 * np.abs(dp_w) + 1e-12
    assert within[both].mean() > 0.999
    big = np.abs(dp_w) > 2000 * ulp
    checked = 0
    for name, (a, b) in dict(means=(0, 3), scales=(3, 6), quats=(6, 10), opacity=(10, 11), sh_dc=(11, 14),
                             sh_rest=(14, 59)).items():
        sb = big[both, a:b]
        if sb.sum() > 50:
            assert rel_l2(dp_g[both, a:b][sb], dp_w[both, a:b][sb]) <= 1e-3, name
            checked += 1
        assert rel_l2(join(mv.m)[both, a:b], mw[both, a:b]) <= 1e-3, name
        assert rel_l2(join(mv.v)[both, a:b], vw[both, a:b]) <= 2e-3, name
    assert checked >= 3
    untouched = ~t_g
    np.testing.assert_array_equal(pg[untouched], p32[untouched])

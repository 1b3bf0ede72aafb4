"""The headline workload at full size, in the launch configuration the bench
times (500k Gaussians, one 1280x720 view, 20 % of the tiles, 85 sampled
pixels per tile, checkpoints every 32 list positions for the warp-per-piece
backward), checked against the oracle on outputs it can compute one by one:
the selection (bit for bit), the projection of every Gaussian, the forward at
512 seeded sampled pixels, the fused loss with the error/age map updates over
every sampled pixel (on the forward's output), the backward of a seeded dL/dI
that is non-zero at those 512 pixels only (so that both sides sum the same
terms), and the fused projection adjoint + hybrid update (mode 1) of the
Gaussians it touches."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu
MARGIN = 1e-4
W, H, N = 1280, 720, 500_000
N_SEL, N_PIX = 720, 85


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_full_size_step_against_oracle(orc):
    from paper_2606_15924_gb300 import binding as B
    from gpu_util import bin_dev, dev, empty_projected, gaussians_dev, projected_host, select_dev, select_host
    B.device_check()
    g = scenes.gaussians(N, seed=scenes.SEED_SCENE, extent=5.0)
    cam = scenes.look_at((0.0, 0.0, -15.0), width=W, height=H, fov_x_deg=60.0)
    err, age = scenes.error_map(W, H, seed=21), scenes.age_map(W, H, seed=22)
    # selection, bit for bit
    sel = select_dev(B, err, age, W, H, N_SEL, N_PIX, seed=7, it=3)
    sel_o = orc.select(err, age, W, H, n_select=N_SEL, n_pix=N_PIX, seed=7, it=3)
    sh = select_host(sel)
    np.testing.assert_array_equal(sh["active_tiles"], sel_o["active_tiles"])
    np.testing.assert_array_equal(sh["pix_idx"], sel_o["pix_idx"])
    # projection of every Gaussian
    gd = gaussians_dev(g)
    pd = empty_projected(N)
    B.project_gaussians(gd, cam, sel["tile_rank"], pd)
    g64 = {k: v.astype(np.float64) for k, v in g.items()}
    prw = orc.project(g64, cam, tile_rank=sel_o["tile_rank"])
    got = projected_host(pd)
    sure_g = prw["margin"] > MARGIN
    assert sure_g.mean() > 0.99
    np.testing.assert_array_equal(got["radius"][sure_g], prw["radius"][sure_g])
    m = sure_g & (prw["radius"] > 0)
    assert m.sum() > 100_000
    np.testing.assert_allclose(got["xy"][m], prw["xy"][m], rtol=1e-5, atol=1e-3)
    np.testing.assert_allclose(got["rgb"][m], prw["rgb"][m], atol=1e-5)
    # binning and the forward with checkpoints, as the trainer runs them
    binned = bin_dev(B, pd, N, cam, sel["tile_rank"], sel["n_sel"], capacity=4_000_000, want_keys=False)
    I = int(binned["n_isect"].item())
    assert 0 < I < 4_000_000
    P = int(sh["pix_off"][-1])
    slots = 64
    rgb = torch.zeros(P, 3, device="cuda")
    T = torch.zeros(P, device="cuda")
    n_last = torch.zeros(P, dtype=torch.int32, device="cuda")
    ck_data = torch.empty(B.checkpoint_bytes(N_SEL, N_PIX, slots) // 4, device="cuda")
    tl = torch.zeros(N_SEL, dtype=torch.int32, device="cuda")
    ck = B.checkpoints(ck_data, slots, N_SEL * N_PIX, rgb, tl)
    B.render_sampled(pd, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"], sel["n_sel"],
                     sel["pix_off"], sel["pix_idx"], N_PIX, cam, (0.0, 0.0, 0.0), rgb, T, n_last, ckpt=ck)
    rng = np.random.default_rng(11)
    S = np.sort(rng.choice(P, 512, replace=False))
    pix = orc.pixel_coords(sel_o["active_tiles"], sel_o["pix_off"], sel_o["pix_idx"], W)[S]
    want = orc.render_pixels(prw, W, H, pix)
    sure_p = want["margin"] > MARGIN
    assert sure_p.mean() > 0.95
    np.testing.assert_array_equal(n_last.cpu().numpy()[S][sure_p], want["n_last"][sure_p])
    assert np.abs(rgb.cpu().numpy()[S][sure_p] - want["rgb"][sure_p]).max() <= 1e-4
    assert np.abs(T.cpu().numpy()[S][sure_p] - want["T"][sure_p]).max() <= 1e-4
    # the fused loss (Sec. 3.7 Eqs. 9-11; App. A) with the error EMA and age updates (Sec. 3.3,
    # Eqs. 2-4) over all of the step's sampled pixels, on the forward's own output
    tgt = scenes.smooth_image(W, H, seed=31)
    err_d, age_d = dev(err), dev(age)
    dLl = torch.zeros(P, 3, device="cuda")
    lam = torch.zeros(N_SEL, device="cuda")
    e_pix = torch.zeros(P, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.loss_sparse_ncc(rgb, dev(tgt), W, H, sel["active_tiles"], sel["n_active"], sel["n_sel"], sel["pix_off"],
                      sel["pix_idx"], N_PIX, (1e-3, 1e-8, 0.4), err_d, age_d, dLl, lam, e_pix, loss)
    rgb_h = rgb.cpu().numpy().astype(np.float64)
    lo = orc.loss(W, H, sel_o, rgb_h, tgt.astype(np.float64), err_f16_bits=err, age=age)
    assert float(loss.item()) == pytest.approx(lo["loss"], rel=1e-5)
    np.testing.assert_allclose(lam.cpu().numpy()[:len(lo["lam"])], lo["lam"], rtol=1e-4, atol=1e-7)
    np.testing.assert_allclose(e_pix.cpu().numpy(), lo["err"], atol=1e-6)
    assert rel_l2(dLl.cpu().numpy(), lo["dL_drgb"]) <= 1e-4
    np.testing.assert_array_equal(age_d.cpu().numpy(), lo["age_map"])   # ages exactly
    got_e = err_d.cpu().numpy().view(np.float16).astype(np.float64)
    want_e = lo["err_map"].view(np.float16).astype(np.float64)
    ulp = np.spacing(np.abs(want_e).astype(np.float16)).astype(np.float64)
    assert np.all(np.abs(got_e - want_e) <= ulp)                         # one fp16 ulp
    # the backward from the checkpoints, dL/dI seeded and non-zero at S only
    dL = np.zeros((P, 3), np.float32)
    dL[S] = rng.normal(0.0, 1e-3, (len(S), 3)).astype(np.float32)
    grad2d = torch.zeros(N, 12, device="cuda")
    B.render_backward_sampled(pd, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"],
                              sel["n_sel"], sel["pix_off"], sel["pix_idx"], N_PIX, cam, (0.0, 0.0, 0.0), T, n_last,
                              dev(dL), grad2d, ckpt=ck)
    g2w = orc.render_backward(prw, W, H, pix, dL[S].astype(np.float64))
    g2g = grad2d.cpu().numpy()
    touched = np.abs(g2w).sum(1) > 0
    assert touched.sum() > 1000
    ok = sure_g
    for c in range(9):
        assert rel_l2(g2g[ok, c], g2w[ok, c]) <= 1e-3, (c, rel_l2(g2g[ok, c], g2w[ok, c]))

    # the projection adjoint fused with the hybrid update (diagonal LM, mode 1), as the step runs it
    gw = orc.project_backward(g64, cam, g2w, tile_rank=sel_o["tile_rank"])        # [N, 59]
    cfg = np.array([1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4, 0.9, 0.999, 1e-15, 1e-8])
    opt = dict(lr=cfg[:6], beta1=cfg[6], beta2=cfg[7], eps_adam=cfg[8], eps_lm=cfg[9], mode=1)
    step = 4
    p0 = np.concatenate([g["means"], g["log_scales"], g["quats"], g["opacity_logits"][:, None],
                         np.asarray(g["sh"]).reshape(N, 48)], 1).astype(np.float32)
    m0 = rng.normal(0.0, 1e-4, p0.shape).astype(np.float32)
    v0 = rng.uniform(1e-8, 1e-6, p0.shape).astype(np.float32)
    t_w = (np.abs(g2w).sum(1) > 0) & (prw["radius"] > 0)
    pw, mw, vw = orc.hybrid_step(p0.astype(np.float64), gw, m0.astype(np.float64), v0.astype(np.float64),
                                 t_w.astype(np.uint8), step, 1, cfg)

    def split(a):
        a = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        return dict(means=a[:, 0:3].contiguous(), log_scales=a[:, 3:6].contiguous(), quats=a[:, 6:10].contiguous(),
                    opacity_logits=a[:, 10].contiguous(), sh=a[:, 11:59].contiguous().view(N, 16, 3))

    def join(d):
        return np.concatenate([d["means"].cpu().numpy(), d["log_scales"].cpu().numpy(), d["quats"].cpu().numpy(),
                               d["opacity_logits"].cpu().numpy()[:, None], d["sh"].cpu().numpy().reshape(N, 48)], 1)

    P_, M_, V_ = split(p0), split(m0), split(v0)
    touched = torch.zeros(N, dtype=torch.uint8, device="cuda")
    adj = B.MultiAdjoint([cam], [pd["radius"]], [grad2d])
    B.project_backward_update(P_, adj, M_, V_, touched, opt, step)
    torch.cuda.synchronize()
    t_g = touched.cpu().numpy().astype(bool)
    both = t_g & t_w & sure_g
    assert both.sum() > 1000 and (t_g[sure_g] == t_w[sure_g]).mean() > 0.999
    # parameters are stored in fp32: the update lands rounded to the parameter's ulp, which for
    # means of a few units is a visible share of a step of ~1e-4; the step is compared where it
    # is well above that rounding, and every element within the rounding plus the gradient's
    # own tolerance
    pg = join(P_).astype(np.float64)
    dp_g, dp_w = pg - p0, pw - p0
    ulp = np.spacing(np.abs(pw).astype(np.float32)).astype(np.float64)
    within = np.abs(pg - pw) <= 1.5 * ulp + 2e-3 * np.abs(dp_w) + 1e-12
    assert within[both].mean() > 0.999
    big = np.abs(dp_w) > 2000 * ulp
    checked = 0
    for name, (a, b) in dict(means=(0, 3), scales=(3, 6), quats=(6, 10), opacity=(10, 11), sh_dc=(11, 14),
                             sh_rest=(14, 59)).items():
        sel_b = big[both, a:b]
        if sel_b.sum() > 100:
            e = rel_l2(dp_g[both, a:b][sel_b], dp_w[both, a:b][sel_b])
            assert e <= 1e-3, (name, e)
            checked += 1
        assert rel_l2(join(M_)[both, a:b], mw[both, a:b]) <= 1e-3, name
    assert checked >= 3
    untouched = ~t_g
    np.testing.assert_array_equal(join(P_)[untouched], p0[untouched])

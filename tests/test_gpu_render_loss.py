"""GPU parity of the floating-point steps against the oracle: projection,
sparse forward rendering, the fused loss with error/age updates, the sparse
backward and the hybrid step.  Tolerances (from the arithmetic): images and
per-pixel values max-abs <= 1e-4; gradients relative L2 <= 1e-3.  Discrete
decisions that floating point takes (culling, radius, alpha thresholds,
termination) are compared exactly except where the oracle's double-precision
value lies within 1e-4 (relative) of the threshold, where either side of it is
a correct single-precision result; those cases are counted and must be rare."""
import numpy as np
import pytest
import torch

import oracle as orc_mod
from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu
MARGIN = 1e-4


@pytest.fixture(scope="module")
def B():
    from paper_2606_15924_gb300 import binding
    binding.device_check()
    return binding


def _c0(seed=0, n=10000):
    g = scenes.gaussians(n, seed=seed)
    cam = scenes.look_at((0.0, 0.0, -4.0), width=256, height=256)
    return g, cam


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("masked", [False, True])
def test_project_parity(B, orc, masked):
    from gpu_util import dev, empty_projected, gaussians_dev, projected_host, tile_count
    g, cam = _c0()
    g["means"][:50, 2] = -4.5                # behind the camera
    g["log_scales"][50:60] = 1.0             # huge splats
    n = len(g["opacity_logits"])
    rank = None
    if masked:
        T = tile_count(256, 256)
        act = np.random.default_rng(2).uniform(size=T) < 0.25
        rank = np.where(act, np.cumsum(act) - 1, -1).astype(np.int32)
    out = empty_projected(n)
    B.project_gaussians(gaussians_dev(g), cam, None if rank is None else dev(rank), out)
    got = projected_host(out)
    want = orc.project({k: v.astype(np.float64) for k, v in g.items()}, cam, tile_rank=rank)
    sure = want["margin"] > MARGIN
    assert sure.mean() > 0.99
    vis_w, vis_g = want["radius"] > 0, got["radius"] > 0
    np.testing.assert_array_equal(vis_w[sure], vis_g[sure])
    np.testing.assert_array_equal(want["radius"][sure], got["radius"][sure])
    m = sure & vis_w
    assert m.sum() > 1000 if not masked else m.sum() > 200
    np.testing.assert_allclose(got["xy"][m], want["xy"][m], rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(got["depth"][m], want["depth"][m], rtol=1e-6)
    np.testing.assert_allclose(got["conic"][m], want["conic"][m], rtol=2e-4, atol=1e-6)
    np.testing.assert_allclose(got["opac"][m], want["opac"][m], atol=1e-6)
    np.testing.assert_allclose(got["rgb"][m], want["rgb"][m], atol=1e-5)
    assert np.all(got["radius"][~vis_g] == 0)


def _render_case(B, orc, pr_np, W, H, n_select, n_pix, seed=3, bg=(0.0, 0.0, 0.0)):
    """GPU select -> bin -> render on given splats; oracle render on the same
    sampled pixels (the sampled set itself is pinned bit-exactly elsewhere, and
    is produced here by the oracle on the same inputs, so both sides render the
    same pixels)."""
    from gpu_util import bin_dev, dev, projected_dev, render_dev, select_dev, select_host
    err = scenes.error_map(W, H, seed=seed)
    age = scenes.age_map(W, H, seed=seed)
    sel = select_dev(B, err, age, W, H, n_select, n_pix, seed=seed)
    sel_o = orc.select(err, age, W, H, n_select=n_select, n_pix=n_pix, seed=seed)
    sel_h = select_host(sel)
    np.testing.assert_array_equal(sel_h["pix_idx"], sel_o["pix_idx"])
    pd = projected_dev(pr_np)
    n = len(pr_np["radius"])
    ref = orc.bin_tiles(pr_np["xy"], pr_np["radius"], pr_np["depth"], W, H, sel_o["tile_rank"])
    scam = dict(viewmat=np.eye(4), fx=1.0, fy=1.0, cx=0, cy=0, width=W, height=H, znear=0.2)
    binned = bin_dev(B, pd, n, scam, sel["tile_rank"], sel["n_sel"], capacity=len(ref[1]) + 64)
    out = render_dev(B, pd, binned, sel, n_pix, scam, bg=bg)
    P = int(sel_o["pix_off"][-1])
    pix = orc.pixel_coords(sel_o["active_tiles"], sel_o["pix_off"], sel_o["pix_idx"], W)
    want = orc.render_pixels({k: np.asarray(v, np.float64) if k != "radius" else v for k, v in pr_np.items()},
                             W, H, pix, bg=bg)
    got = dict(rgb=out["rgb"][:P].cpu().numpy(), T=out["T"][:P].cpu().numpy(),
               n_last=out["n_last"][:P].cpu().numpy())
    return got, want, sel, sel_o, binned, pd, out


@pytest.mark.parametrize("W,H,n,n_select,n_pix", [(256, 256, 4000, 64, 256), (256, 256, 4000, 256, 256),
                                                   (200, 130, 3000, 30, 84), (640, 360, 20000, 180, 25)])
def test_render_parity_synthetic_splats(B, orc, W, H, n, n_select, n_pix):
    pr = scenes.projected(n, W, H, seed=n)
    got, want, *_ = _render_case(B, orc, pr, W, H, n_select, n_pix, bg=(0.1, 0.2, 0.3))
    sure = want["margin"] > MARGIN
    assert sure.mean() > 0.98
    assert (want["n_contrib"] > 2).mean() > 0.5
    np.testing.assert_array_equal(got["n_last"][sure], want["n_last"][sure])
    assert np.abs(got["rgb"][sure] - want["rgb"][sure]).max() <= 1e-4
    assert np.abs(got["T"][sure] - want["T"][sure]).max() <= 1e-4


def test_full_mask_equals_dense_bitwise(B, orc):
    """The sampled path at every pixel is the dense render; any subset of
    tiles/pixels reproduces the dense values at those pixels bit for bit."""
    W, H = 256, 256
    pr = scenes.projected(4000, W, H, seed=77)
    d_got, d_want, d_sel, d_sel_o, *_ = _render_case(B, orc, pr, W, H, 256, 256)
    s_got, s_want, s_sel, s_sel_o, *_ = _render_case(B, orc, pr, W, H, 64, 84)
    dpix = orc.pixel_coords(d_sel_o["active_tiles"], d_sel_o["pix_off"], d_sel_o["pix_idx"], W)
    spix = orc.pixel_coords(s_sel_o["active_tiles"], s_sel_o["pix_off"], s_sel_o["pix_idx"], W)
    img = np.zeros((H, W, 3), np.float32)
    img[dpix[:, 1], dpix[:, 0]] = d_got["rgb"]
    np.testing.assert_array_equal(img[spix[:, 1], spix[:, 0]], s_got["rgb"])


def test_forward_blend_variants_bitwise(B, orc):
    """The forward picks its blend by how many warps the launch has (selects
    for a sparse launch, branches for a dense one); both give the same bits.
    The same 64 active tiles are rendered once with n_active_max = 64 and
    once with an upper bound large enough for the branch variant (the blocks
    past n_active exit at once)."""
    from gpu_util import bin_dev, dev, projected_dev, select_dev
    W = H = 256
    pr = scenes.projected(4000, W, H, seed=91)
    err, age = scenes.error_map(W, H), scenes.age_map(W, H)
    n_pix = 256
    sel = select_dev(B, err, age, W, H, 64, n_pix, seed=5)
    pd = projected_dev(pr)
    cam = dict(viewmat=np.eye(4), fx=100.0, fy=100.0, cx=W / 2, cy=H / 2, width=W, height=H, znear=0.2)
    binned = bin_dev(B, pd, 4000, cam, sel["tile_rank"], sel["n_sel"], capacity=300000)
    outs = []
    for n_active_max in (sel["n_sel"], 20000):   # 20000 blocks x 8 warps: many warps per SM
        P = sel["n_sel"] * n_pix
        o = dict(rgb=torch.zeros(P, 3, device="cuda"), T=torch.zeros(P, device="cuda"),
                 n_last=torch.zeros(P, dtype=torch.int32, device="cuda"))
        B.render_sampled(pd, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"], n_active_max,
                         sel["pix_off"], sel["pix_idx"], n_pix, cam, (0.1, 0.2, 0.3), o["rgb"], o["T"], o["n_last"])
        outs.append(o)
    torch.cuda.synchronize()
    for k in ("rgb", "T", "n_last"):
        assert torch.equal(outs[0][k], outs[1][k]), k


def test_render_chain_from_gaussians(B, orc):
    """Raw Gaussians of the tiny configuration through project -> bin ->
    render on the GPU against the oracle's double-precision chain."""
    from gpu_util import bin_dev, empty_projected, gaussians_dev, render_dev, select_dev
    g, cam = _c0(seed=0)
    W = H = 256
    for n_select, n_pix in ((256, 256), (64, 256)):
        err, age = scenes.error_map(W, H), scenes.age_map(W, H)
        sel = select_dev(B, err, age, W, H, n_select, n_pix, seed=1)
        sel_o = orc.select(err, age, W, H, n_select=n_select, n_pix=n_pix, seed=1)
        pd = empty_projected(10000)
        B.project_gaussians(gaussians_dev(g), cam, sel["tile_rank"], pd)
        binned = bin_dev(B, pd, 10000, cam, sel["tile_rank"], sel["n_sel"], capacity=400000)
        out = render_dev(B, pd, binned, sel, n_pix, cam)
        prw = orc.project({k: v.astype(np.float64) for k, v in g.items()}, cam, tile_rank=sel_o["tile_rank"])
        pix = orc.pixel_coords(sel_o["active_tiles"], sel_o["pix_off"], sel_o["pix_idx"], W)
        want = orc.render_pixels(prw, W, H, pix)
        P = len(pix)
        rgb = out["rgb"][:P].cpu().numpy()
        # a splat whose radius or tile rectangle sits at a threshold may be
        # listed in its boundary tiles on one side and not on the other: the
        # pixels of that ring of tiles that it reaches with a visible alpha are
        # excluded
        amb = want["margin"] <= MARGIN
        geo = orc.project({k: v.astype(np.float64) for k, v in g.items()}, cam)
        bad_g = np.nonzero((prw["margin"] <= MARGIN) | (geo["margin"] <= MARGIN))[0]
        ptx, pty = pix[:, 0] // 16, pix[:, 1] // 16
        for i in bad_g:
            if geo["radius"][i] <= 0:
                continue
            r = float(geo["radius"][i])
            x, y = geo["xy"][i]

            def covered(rr):
                return ((ptx >= np.floor((x - rr) / 16)) & (ptx <= np.floor((x + rr) / 16))
                        & (pty >= np.floor((y - rr) / 16)) & (pty <= np.floor((y + rr) / 16)))
            ring = covered(r + 1.01) & ~covered(r - 1.01)
            dx, dy = pix[:, 0] + 0.5 - x, pix[:, 1] + 0.5 - y
            a, b, c = geo["conic"][i]
            alpha = geo["opac"][i] * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
            amb |= ring & (alpha >= 0.5 / 255)
        assert amb.mean() < 0.02
        err_max = np.abs(rgb[~amb] - want["rgb"][~amb]).max()
        assert err_max <= 1e-4, err_max


def _loss_inputs(W, H, n_select, n_pix, seed):
    err = scenes.error_map(W, H, seed=seed)
    age = scenes.age_map(W, H, seed=seed, max_age=65535)
    target = scenes.smooth_image(W, H, seed=seed + 1)
    return err, age, target


@pytest.mark.parametrize("structure", ["ncc", "ssim"])
@pytest.mark.parametrize("W,H,n_select,n_pix", [(256, 256, 64, 256), (200, 130, 40, 25), (1280, 720, 720, 84),
                                                 (64, 48, 12, 1)])
def test_loss_parity(B, orc, W, H, n_select, n_pix, structure):
    """The fused loss with its error/age map updates against the oracle's;
    structure: the sparse NCC term (Sec. 3.7) or Table 4's S-SSIM variant."""
    from gpu_util import dev, select_dev, select_host
    err, age, target = _loss_inputs(W, H, n_select, n_pix, seed=W)
    sel = select_dev(B, err, age, W, H, n_select, n_pix, seed=9)
    sh = select_host(sel)
    P = int(sh["pix_off"][-1])
    A = sh["n_active"]
    rgb = np.random.default_rng(4).uniform(0, 1, (max(P, 1), 3)).astype(np.float32)
    rgb[:P] = 0.7 * target[orc.pixel_coords(sh["active_tiles"], sh["pix_off"], sh["pix_idx"], W)[:, 1],
                           orc.pixel_coords(sh["active_tiles"], sh["pix_off"], sh["pix_idx"], W)[:, 0]] + 0.3 * rgb[:P]
    err_d, age_d = dev(err), dev(age)
    dL = torch.zeros(max(P, 1), 3, device="cuda")
    lam = torch.zeros(max(sel["n_sel"], 1), device="cuda")
    e = torch.zeros(max(P, 1), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.loss_sparse_ncc(dev(rgb), dev(target), W, H, sel["active_tiles"], sel["n_active"], sel["n_sel"],
                      sel["pix_off"], sel["pix_idx"], n_pix, (1e-3, 1e-8, 0.4), err_d, age_d, dL, lam, e, loss,
                      structure=structure)
    oloss = orc.loss if structure == "ncc" else orc.loss_ssim
    want = oloss(W, H, sh, rgb[:P].astype(np.float64), target.astype(np.float64), err_f16_bits=err, age=age)
    assert float(loss.item()) == pytest.approx(want["loss"], rel=1e-5)
    np.testing.assert_allclose(lam[:A].cpu().numpy(), want["lam"], rtol=1e-4, atol=1e-7)
    np.testing.assert_allclose(e[:P].cpu().numpy(), want["err"], atol=1e-6)
    assert rel_l2(dL[:P].cpu().numpy(), want["dL_drgb"]) <= 1e-4
    assert np.abs(dL[:P].cpu().numpy() - want["dL_drgb"]).max() <= 1e-4 * np.abs(want["dL_drgb"]).max() + 1e-9
    np.testing.assert_array_equal(age_d.cpu().numpy(), want["age_map"])
    got_e = err_d.cpu().numpy().view(np.float16).astype(np.float64)
    want_e = want["err_map"].view(np.float16).astype(np.float64)
    ulp = np.spacing(np.abs(want_e).astype(np.float16)).astype(np.float64)
    assert np.all(np.abs(got_e - want_e) <= ulp)     # one fp16 ulp


@pytest.mark.parametrize("split", [False, True])
def test_backward_parity(B, orc, split):
    """grad2d and the parameter gradients of the tiny scene against the
    oracle's analytic backward (relative L2 <= 1e-3 per parameter group);
    split: the backward replays each tile list in pieces of 32 positions from
    the forward's checkpoints (few slots, so that a long tail piece occurs, or
    the trainer's 64), at 1, 3, 5 and 8 pixels per lane."""
    from gpu_util import bin_dev, dev, empty_projected, gaussians_dev, render_dev, select_dev, select_host
    g, cam = _c0(seed=5, n=3000)
    g["log_scales"] += 1.0
    W = H = 256
    n = 3000
    err, age = scenes.error_map(W, H), scenes.age_map(W, H)
    target = scenes.smooth_image(W, H, seed=2)
    # n_pix 25, 84, 150, 256: 1, 3, 5 and 8 pixels per lane in the warp-per-piece backward
    for n_select, n_pix in ((64, 84), (256, 256), (64, 25), (64, 150)):
        sel = select_dev(B, err, age, W, H, n_select, n_pix, seed=4)
        sh = select_host(sel)
        gd = gaussians_dev(g)
        pd = empty_projected(n)
        B.project_gaussians(gd, cam, sel["tile_rank"], pd)
        binned = bin_dev(B, pd, n, cam, sel["tile_rank"], sel["n_sel"], capacity=300000)
        out = render_dev(B, pd, binned, sel, n_pix, cam)
        ck = None
        if split:
            every = 32                                        # list positions per slot
            longest = int(out["n_last"].max().item())
            assert longest > 4 * every                        # several pieces
            # few slots (a long tail piece past them) or as many as the trainer uses
            slots = 3 if n_pix in (25, 84) else 64
            stride = sel["n_sel"] * n_pix
            ck_data = torch.full((B.checkpoint_bytes(sel["n_sel"], n_pix, slots) // 4,), float("nan"),
                                 device="cuda")
            # the second case also has the forward record each tile's longest run
            tl = torch.full((sel["n_sel"],), -1, dtype=torch.int32, device="cuda") if n_pix in (150, 256) else None
            ck = B.checkpoints(ck_data, slots, stride, out["rgb"], tl)
            B.render_sampled(pd, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"],
                             sel["n_sel"], sel["pix_off"], sel["pix_idx"], n_pix, cam, (0.0, 0.0, 0.0), out["rgb"],
                             out["T"], out["n_last"], ckpt=ck)
        P = int(sh["pix_off"][-1])
        pix = orc.pixel_coords(sh["active_tiles"], sh["pix_off"], sh["pix_idx"], W)
        # one dL/dI drives both sides (a seeded input, not computed by either)
        dLd = np.random.default_rng(8).normal(0, 1e-3, (P, 3)).astype(np.float32)
        grad2d = torch.zeros(n, 12, device="cuda")
        grads = {k: torch.zeros_like(v) for k, v in gd.items()}
        touched = torch.zeros(n, dtype=torch.uint8, device="cuda")
        B.backward_sampled(gd, cam, pd, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"],
                           sel["n_sel"], sel["pix_off"], sel["pix_idx"], n_pix, (0.0, 0.0, 0.0), out["T"],
                           out["n_last"], dev(dLd), grad2d, grads, touched, ckpt=ck)
        if split and tl is not None:   # the recorded runs are the per-tile maxima of n_last
            nl = out["n_last"].cpu().numpy()
            off = sh["pix_off"]
            want_tl = [int(nl[off[r]:off[r + 1]].max(initial=0)) for r in range(len(off) - 1)]
            np.testing.assert_array_equal(tl.cpu().numpy()[:len(want_tl)], want_tl)
        g64 = {k: v.astype(np.float64) for k, v in g.items()}
        prw = orc.project(g64, cam, tile_rank=sh["tile_rank"])
        g2w = orc.render_backward(prw, W, H, pix, dLd.astype(np.float64))
        gw = orc.project_backward(g64, cam, g2w, tile_rank=sh["tile_rank"])
        g2g = grad2d.cpu().numpy()
        col = [0, 1, 2, 3, 4, 5, 6, 7, 8]
        # exclude splats with a decision at a threshold (their gradient may legitimately differ)
        ok = prw["margin"] > MARGIN
        for c in col:
            assert rel_l2(g2g[ok, c], g2w[ok, c]) <= 1e-3, (c, rel_l2(g2g[ok, c], g2w[ok, c]))
        gg = np.concatenate([grads["means"].cpu().numpy(), grads["log_scales"].cpu().numpy(),
                             grads["quats"].cpu().numpy(), grads["opacity_logits"].cpu().numpy()[:, None],
                             grads["sh"].cpu().numpy().reshape(n, 48)], 1)
        for name, (a, b) in dict(means=(0, 3), scales=(3, 6), quats=(6, 10), opacity=(10, 11), sh_dc=(11, 14),
                                 sh_rest=(14, 59)).items():
            assert rel_l2(gg[ok, a:b], gw[ok, a:b]) <= 1e-3, (name, rel_l2(gg[ok, a:b], gw[ok, a:b]))
        t_w = (np.abs(g2w).sum(1) > 0) & (prw["radius"] > 0)
        np.testing.assert_array_equal(touched.cpu().numpy().astype(bool)[ok], t_w[ok])


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_hybrid_step_parity(B, orc, mode):
    n = 5000
    rng = np.random.default_rng(mode)
    p = rng.normal(size=(n, 59)).astype(np.float32)
    g = rng.normal(scale=0.05, size=(n, 59)).astype(np.float32)
    m = rng.normal(scale=0.01, size=(n, 59)).astype(np.float32)
    v = rng.uniform(1e-6, 1e-3, size=(n, 59)).astype(np.float32)
    touched = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    cfg = np.array([1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4, 0.9, 0.999, 1e-15, 1e-8])

    def split(a):
        a = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        return dict(means=a[:, 0:3].contiguous(), log_scales=a[:, 3:6].contiguous(), quats=a[:, 6:10].contiguous(),
                    opacity_logits=a[:, 10].contiguous(), sh=a[:, 11:59].contiguous().view(n, 16, 3))

    def join(d):
        return np.concatenate([d["means"].cpu().numpy(), d["log_scales"].cpu().numpy(), d["quats"].cpu().numpy(),
                               d["opacity_logits"].cpu().numpy()[:, None], d["sh"].cpu().numpy().reshape(n, 48)], 1)

    P_, G_, M_, V_ = split(p), split(g), split(m), split(v)
    opt = dict(lr=cfg[:6], beta1=cfg[6], beta2=cfg[7], eps_adam=cfg[8], eps_lm=cfg[9], mode=mode)
    B.hybrid_step(P_, G_, M_, V_, n, torch.from_numpy(touched).cuda(), None, 0, 7, opt)
    pw, mw, vw = orc.hybrid_step(p, g, m, v, touched, 7, mode, cfg)
    # fp32 rounding of b1 m and (1 - b1) g (|m|, |g| ~ 1e-2) is ~1e-9 absolute
    np.testing.assert_allclose(join(M_), mw, rtol=1e-5, atol=2e-8)
    np.testing.assert_allclose(join(V_), vw, rtol=1e-5, atol=1e-10)
    dp_g, dp_w = join(P_) - p, pw - p
    assert rel_l2(dp_g, dp_w) <= 1e-3
    np.testing.assert_allclose(join(P_), pw, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("n_select,n_pix", [(64, 84), (256, 256)])
def test_error_stats_parity(B, orc, n_select, n_pix):
    """Sec. 3.8 error back-projection statistics (sum e w, sum w, sum D w per
    Gaussian) against the oracle, from a seeded per-pixel error that both
    sides take as input; with accumulate the second call adds to the first."""
    from gpu_util import bin_dev, dev, empty_projected, gaussians_dev, render_dev, select_dev, select_host
    g, cam = _c0(seed=5, n=3000)
    g["log_scales"] += 1.0
    W = H = 256
    n = 3000
    err, age = scenes.error_map(W, H), scenes.age_map(W, H)
    sel = select_dev(B, err, age, W, H, n_select, n_pix, seed=4)
    sh = select_host(sel)
    gd = gaussians_dev(g)
    pd = empty_projected(n)
    B.project_gaussians(gd, cam, sel["tile_rank"], pd)
    binned = bin_dev(B, pd, n, cam, sel["tile_rank"], sel["n_sel"], capacity=300000)
    out = render_dev(B, pd, binned, sel, n_pix, cam)
    P = int(sh["pix_off"][-1])
    pix = orc.pixel_coords(sh["active_tiles"], sh["pix_off"], sh["pix_idx"], W)
    e = np.random.default_rng(9).uniform(0.0, 2.0, P).astype(np.float32)
    stats = torch.zeros(n, 4, device="cuda")
    args = (pd, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"], sel["n_sel"], sel["pix_off"],
            sel["pix_idx"], n_pix, cam, out["n_last"], dev(e))
    B.error_stats_sampled(*args, stats)
    torch.cuda.synchronize()
    got = stats.cpu().numpy().astype(np.float64)
    g64 = {k: v.astype(np.float64) for k, v in g.items()}
    prw = orc.project(g64, cam, tile_rank=sh["tile_rank"])
    want = orc.error_stats(prw, W, H, pix, e.astype(np.float64))
    ok = prw["margin"] > MARGIN
    assert (want[ok, 1] > 0).sum() > 200
    for c in range(3):
        assert rel_l2(got[ok, c], want[ok, c]) <= 1e-3, (c, rel_l2(got[ok, c], want[ok, c]))
    assert np.all(got[:, 3] == 0.0)
    B.error_stats_sampled(*args, stats, accumulate=True)
    torch.cuda.synchronize()
    # float atomics sum in a different order on each call: equal up to rounding
    np.testing.assert_allclose(stats.cpu().numpy()[:, :3], 2.0 * got[:, :3], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("split", [False, True])
def test_statistics_fused_into_backward(B, orc, split):
    """Eq. 12's statistics accumulated inside the backward replay
    (render_backward_sampled_stats) against the oracle; the gradients equal
    those of the plain backward; accumulate adds a second call's sums.
    split: the warp-per-piece replay from checkpoints (the sums ride on it);
    otherwise the whole-tile backward followed by the statistics pass."""
    from gpu_util import bin_dev, dev, empty_projected, gaussians_dev, select_dev, select_host
    g, cam = _c0(seed=5, n=3000)
    g["log_scales"] += 1.0
    W = H = 256
    n = 3000
    n_select, n_pix = 64, 85
    err, age = scenes.error_map(W, H), scenes.age_map(W, H)
    sel = select_dev(B, err, age, W, H, n_select, n_pix, seed=4)
    sh = select_host(sel)
    pd = empty_projected(n)
    B.project_gaussians(gaussians_dev(g), cam, sel["tile_rank"], pd)
    binned = bin_dev(B, pd, n, cam, sel["tile_rank"], sel["n_sel"], capacity=300000)
    Pm = sel["n_sel"] * n_pix
    rgb, T = torch.zeros(Pm, 3, device="cuda"), torch.zeros(Pm, device="cuda")
    n_last = torch.zeros(Pm, dtype=torch.int32, device="cuda")
    ck = None
    if split:
        slots = 64
        data = torch.empty(B.checkpoint_bytes(sel["n_sel"], n_pix, slots) // 4, device="cuda")
        ck = B.checkpoints(data, slots, Pm, rgb, torch.zeros(sel["n_sel"], dtype=torch.int32, device="cuda"))
    B.render_sampled(pd, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"], sel["n_sel"],
                     sel["pix_off"], sel["pix_idx"], n_pix, cam, (0.0, 0.0, 0.0), rgb, T, n_last, ckpt=ck)
    P = int(sh["pix_off"][-1])
    rng = np.random.default_rng(19)
    e = rng.uniform(0.0, 2.0, Pm).astype(np.float32)
    dL = rng.normal(0.0, 1e-3, (Pm, 3)).astype(np.float32)
    args = (pd, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"], sel["n_sel"], sel["pix_off"],
            sel["pix_idx"], n_pix, cam, (0.0, 0.0, 0.0), T, n_last, dev(dL))
    g_plain = torch.zeros(n, 12, device="cuda")
    B.render_backward_sampled(*args, g_plain, ckpt=ck)
    g_fused = torch.zeros(n, 12, device="cuda")
    stats = torch.full((n, 4), 5.0, device="cuda")           # zeroed by the call
    B.render_backward_sampled_stats(*args, g_fused, dev(e), stats, ckpt=ck)
    torch.cuda.synchronize()
    a, b = g_fused.cpu().numpy(), g_plain.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
    got = stats.cpu().numpy().astype(np.float64)
    pix = orc.pixel_coords(sh["active_tiles"], sh["pix_off"], sh["pix_idx"], W)
    prw = orc.project({k: v.astype(np.float64) for k, v in g.items()}, cam, tile_rank=sh["tile_rank"])
    want = orc.error_stats(prw, W, H, pix, e[:P].astype(np.float64))
    ok = prw["margin"] > MARGIN
    assert (want[ok, 1] > 0).sum() > 200
    for c in range(3):
        assert rel_l2(got[ok, c], want[ok, c]) <= 1e-3, (c, rel_l2(got[ok, c], want[ok, c]))
    assert np.all(got[:, 3] == 0.0)
    B.render_backward_sampled_stats(*args, g_fused, dev(e), stats, accumulate=True, ckpt=ck)
    torch.cuda.synchronize()
    np.testing.assert_allclose(stats.cpu().numpy()[:, :3], 2.0 * got[:, :3], rtol=1e-5, atol=1e-6)

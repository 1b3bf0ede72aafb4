"""The row layout of the geometric fields (tgs_gaussians::geo_stride: means,
log-scales, opacity logits and quats of a Gaussian in one 64-byte row)
against the four packed arrays: every call that reads or writes them gives
the same bits in either layout - the projection, the projection adjoint (one
view and several), the fused adjoint + update, the hybrid step and density
control - and a trainer whose parameters, gradients and moments are rows
trains like one on packed arrays."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu

KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")
W, H = 256, 192


@pytest.fixture(scope="module")
def B():
    from paper_2606_15924_gb300 import binding
    binding.device_check()
    return binding


def _rows(g, stride=16):
    from paper_2606_15924_gb300.pipeline import as_geo_rows
    return as_geo_rows(g, stride)


def _same(a, b):
    for k in KEYS:
        assert torch.equal(a[k].contiguous(), b[k].contiguous()), k


def _rand_like(g, seed, scale):
    gen = torch.Generator(device="cuda").manual_seed(seed)
    return {k: torch.rand(v.shape, generator=gen, device="cuda") * scale for k, v in g.items()}


def _setup(n=20000):
    from gpu_util import gaussians_dev
    from paper_2606_15924_gb300.batched import MultiViewTrainer
    from paper_2606_15924_gb300.config import Config
    from gpu_util import dev
    g = gaussians_dev(scenes.gaussians(n, seed=0))
    cams = scenes.orbit(3, 4.0, W, H)
    targets = [dev(scenes.smooth_image(W, H, seed=10 + k)) for k in range(3)]
    cfg = Config()
    cfg.opt.mode = 1
    mv = MultiViewTrainer(g, cams, targets, [0.3, 0.6, 0.2], cfg=cfg)
    for k, v in enumerate(mv.views):
        v.err_map.copy_(dev(scenes.error_map(W, H, seed=k).view(np.int16)))
    mv.forward()
    mv.loss_and_maps()
    mv._render_bwd()
    torch.cuda.synchronize()
    return mv


@pytest.mark.parametrize("stride", [12, 16, 20])
def test_projection_same_bits(B, stride):
    from gpu_util import gaussians_dev
    g = gaussians_dev(scenes.gaussians(30000, seed=3))
    r = _rows(g, stride)
    assert r["means"].stride(0) == stride and not r["means"].is_contiguous()
    cam = scenes.look_at((0.0, 0.0, -4.0), width=W, height=H)
    outs = []
    for x in (g, r):
        n = x["means"].shape[0]
        o = dict(xy=torch.zeros(n, 2, device="cuda"), conic_opac=torch.zeros(n, 4, device="cuda"),
                 rgb=torch.zeros(n, 3, device="cuda"), depth=torch.zeros(n, device="cuda"),
                 radius=torch.zeros(n, dtype=torch.int32, device="cuda"))
        B.project_gaussians(x, cam, None, o)
        outs.append(o)
    torch.cuda.synchronize()
    assert int((outs[0]["radius"] > 0).sum()) > 1000
    for k in outs[0]:
        assert torch.equal(outs[0][k], outs[1][k]), k


def test_adjoints_update_and_hybrid_same_bits(B):
    from paper_2606_15924_gb300.pipeline import zeros_like_params
    mv = _setup()
    p0 = {k: mv.params[k].clone() for k in KEYS}
    m0, v0 = _rand_like(p0, 5, 1e-3), _rand_like(p0, 6, 1e-4)
    step = torch.full((1,), 3, dtype=torch.int32, device="cuda")
    res = []
    for layout in ("packed", "rows"):
        conv = (lambda d: {k: v.clone() for k, v in d.items()}) if layout == "packed" else _rows
        p, m, v = conv(p0), conv(m0), conv(v0)
        # several views' adjoint into gradients of the same layout (untouched rows zeroed)
        grads = zeros_like_params(p)
        for k in KEYS:
            grads[k].fill_(7.0)
        t = torch.zeros(mv.n, dtype=torch.uint8, device="cuda")
        B.project_backward_multi(p, mv.adj, grads, t, write_untouched=True)
        # the one-view adjoint
        g1 = zeros_like_params(p)
        t1 = torch.zeros(mv.n, dtype=torch.uint8, device="cuda")
        v1 = mv.views[1]
        B.project_backward(p, v1.ccam, v1.proj, v1.grad2d, g1, t1)
        # the hybrid step on the multi-view gradients, then the fused update on copies
        ph, mh, vh = (conv(x) for x in (p, m, v))
        B.hybrid_step(ph, grads, mh, vh, mv.n, t, None, 0, 1, mv.opt, step_dev=step)
        tf = torch.zeros(mv.n, dtype=torch.uint8, device="cuda")
        B.project_backward_update(p, mv.adj, m, v, tf, mv.opt, 1, step_dev=step)
        torch.cuda.synchronize()
        assert torch.equal(t, tf) and int(t.sum()) > 100
        res.append(dict(grads=grads, g1=g1, t1=t1, ph=ph, mh=mh, vh=vh, pf=p, mf=m, vf=v, t=t))
    a, b = res
    assert torch.equal(a["t"], b["t"]) and torch.equal(a["t1"], b["t1"])
    for k in ("grads", "g1", "ph", "mh", "vh", "pf", "mf", "vf"):
        _same(a[k], b[k])


def test_density_control_same_bits(B):
    from gpu_util import gaussians_dev
    from paper_2606_15924_gb300.pipeline import zeros_like_params
    n = 20000
    g = gaussians_dev(scenes.gaussians(n, seed=4))
    rng = np.random.default_rng(4)
    st = np.zeros((n, 4), np.float32)
    st[:, 1] = rng.uniform(0.01, 3.0, n)
    st[:, 0] = rng.uniform(0, 1, n) * st[:, 1]
    st[:, 2] = rng.uniform(0, 2, n) * st[:, 1]
    ac = np.zeros((n, 2), np.float32)
    ac[:, 1] = rng.integers(1, 5, n)
    ac[:, 0] = rng.exponential(2e-4, n) * ac[:, 1]
    st_d, ac_d = torch.from_numpy(st).cuda(), torch.from_numpy(ac).cuda()
    m0, v0 = _rand_like(g, 7, 1e-3), _rand_like(g, 8, 1e-4)
    cfg = B.density_params(0.56, 2e-4, float(np.log(0.045)), float(np.log(0.005 / 0.995)), topk_permille=700)
    cap = 2 * n
    outs = []
    for layout in ("packed", "rows"):
        conv = (lambda d: {k: v.clone() for k, v in d.items()}) if layout == "packed" else _rows
        p, m, v = conv(g), conv(m0), conv(v0)
        po, mo, vo = (zeros_like_params(x, cap) for x in (p, m, v))
        n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
        src = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        B.density_control(p, m, v, st_d, ac_d, cfg, po, mo, vo, cap, n_out, src)
        torch.cuda.synchronize()
        outs.append((po, mo, vo, int(n_out.item()), src))
    (pa, ma, va, na, sa), (pb, mb, vb, nb, sb) = outs
    assert na == nb and n // 2 < na < 2 * n and torch.equal(sa, sb)
    for x, y in ((pa, pb), (ma, mb), (va, vb)):
        _same({k: t[:na] for k, t in x.items()}, {k: t[:na] for k, t in y.items()})


def test_trainer_on_rows_trains_like_packed(B):
    """Twenty captured steps of the one-view sampled trainer from the same
    start in either layout: the float atomics of the render backward make the
    two runs differ by rounding only."""
    from gpu_util import gaussians_dev
    from paper_2606_15924_gb300.pipeline import Trainer
    g = gaussians_dev(scenes.gaussians(20000, seed=5))
    cam = scenes.look_at((0.0, 0.0, -4.0), width=W, height=H)
    tgt = torch.from_numpy(scenes.smooth_image(W, H, seed=8)).cuda()
    runs = []
    for layout in ("packed", "rows"):
        p = {k: v.clone() for k, v in g.items()} if layout == "packed" else _rows(g)
        tr = Trainer(p, cam, tgt, tile_fraction=0.5, pixel_rate=1 / 3)
        if layout == "rows":
            assert tr.m["means"].stride(0) == 16 and tr.v["quats"].stride(0) == 16
        tr.init_error_map()
        tr.capture()
        losses = []
        for _ in range(20):
            tr.replay()
            losses.append(tr.loss.clone())
        torch.cuda.synchronize()
        runs.append((p, [float(x.item()) for x in losses]))
    (pa, la), (pb, lb) = runs
    np.testing.assert_allclose(la, lb, rtol=1e-4)
    assert la[-1] < la[0]
    for k in KEYS:
        d = (pa[k] - pb[k]).abs().max().item()
        span = (pa[k] - g[k]).abs().max().item()
        assert d <= 1e-2 * span + 1e-6, (k, d, span)

"""The differentiable wrapper (torch.autograd.Function over render_sampled /
backward_sampled): central finite differences (eps 1e-3) on 64 seeded
Gaussians of a 2M-Gaussian 1600x1060 scene, and the gradient of a
2000-Gaussian crop against the double-precision oracle."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu
W, H = 1600, 1060


@pytest.fixture(scope="module")
def mods():
    from paper_2606_15924_gb300 import autograd as AG
    from paper_2606_15924_gb300 import binding as B
    B.device_check()
    return B, AG


def _dev(g):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in g.items()}


def _cam():
    return scenes.look_at((0.0, 0.0, -15.0), width=W, height=H)


def test_finite_differences_2M(mods):
    B, AG = mods
    g_np = scenes.gaussians(2_000_000, seed=21, extent=5.0)
    cam = _cam()
    P = _dev(g_np)
    n = 2_000_000
    proj = dict(xy=torch.zeros(n, 2, device="cuda"), conic_opac=torch.zeros(n, 4, device="cuda"),
                rgb=torch.zeros(n, 3, device="cuda"), depth=torch.zeros(n, device="cuda"),
                radius=torch.zeros(n, dtype=torch.int32, device="cuda"))
    B.project_gaussians(P, cam, None, proj)
    rad = proj["radius"].cpu().numpy()
    opac = proj["conic_opac"][:, 3].cpu().numpy()
    xy = proj["xy"].cpu().numpy()
    rng = np.random.default_rng(5)
    cand = np.nonzero((rad >= 4) & (rad <= 30) & (opac > 0.3) & (xy[:, 0] > 40) & (xy[:, 0] < W - 40)
                      & (xy[:, 1] > 40) & (xy[:, 1] < H - 40))[0]
    chosen = rng.choice(cand, 64, replace=False)
    tx_n = (W + 15) // 16
    EPS = (1e-3, 1e-4)
    fd_all, an_all = {e: [] for e in EPS}, []
    leaf = {k: v.detach().clone().requires_grad_(True) for k, v in P.items()}
    for gi in chosen:
        x, y, r = xy[gi, 0], xy[gi, 1], rad[gi] + 16
        tiles = [ty * tx_n + tx for ty in range(max(0, int((y - r) // 16)), min((H + 15) // 16, int((y + r) // 16) + 1))
                 for tx in range(max(0, int((x - r) // 16)), min(tx_n, int((x + r) // 16) + 1))]
        raster = AG.SampledRaster.from_tiles(cam, n, tiles)
        w = torch.from_numpy(np.random.default_rng(int(gi)).normal(size=(raster.P, 3)).astype(np.float32)).cuda()
        for v in leaf.values():
            v.grad = None
        rgb = AG.render_sampled(leaf, raster)
        (rgb * w).sum().backward()
        an = np.concatenate([leaf["means"].grad[gi].cpu().numpy(), leaf["log_scales"].grad[gi].cpu().numpy(),
                             leaf["quats"].grad[gi].cpu().numpy(), leaf["opacity_logits"].grad[gi:gi + 1].cpu().numpy(),
                             leaf["sh"].grad[gi].reshape(48).cpu().numpy()])
        w64 = w.double()

        def loss(key, idx, delta):
            """loss with one parameter moved in place (restored afterwards);
            returns the loss and the realised float32 parameter value"""
            flat = P[key].view(n, -1)
            orig = flat[gi, idx].clone()
            flat[gi, idx] = orig + delta
            val = float(flat[gi, idx].item())
            with torch.no_grad():
                out = AG.render_sampled(P, raster)
            l = float((out.double() * w64).sum().item())
            flat[gi, idx] = orig
            return l, val

        for eps in EPS:
            fd = []
            for key, cnt in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("sh", 48)):
                for idx in range(cnt):
                    lp, xp = loss(key, idx, eps)
                    lm, xm = loss(key, idx, -eps)
                    fd.append((lp - lm) / (xp - xm))
            fd_all[eps].append(np.array(fd))
        an_all.append(an)
    an_all = np.stack(an_all)
    # Central differences straddle discrete decisions of the method: a pixel
    # crossing alpha = 1/255 (a sub-pixel shift of a splat flips a few of its
    # boundary pixels, each moving the quotient by O(1)), an integer radius or
    # a tile rectangle changing.  The exact double-precision oracle, run with
    # the same procedure on windows of this scene, shows the same statistics:
    # at eps 1e-3 correlation 0.46-1.0 and medians up to ~2 on means, scales
    # and quaternions; at eps 1e-4 scales / quaternions / opacity agree to
    # ~1e-2, means still ~0.3 median (exact only at 1e-5).  The limits below
    # encode that; the strict gradient check is against the oracle (next test).
    groups = dict(means=(0, 3), scales=(3, 6), quats=(6, 10), opacity=(10, 11), sh_dc=(11, 14), sh_rest=(14, 59))
    lim = {1e-3: dict(means=(0.95, None), scales=(0.9, None), quats=(0.9, None), opacity=(0.99, 0.05),
                      sh_dc=(0.999, 0.03), sh_rest=(0.999, 0.03)),
           1e-4: dict(means=(0.95, None), scales=(0.99, 0.05), quats=(0.99, 0.05), opacity=(0.99, 0.1),
                      sh_dc=(0.999, 0.03), sh_rest=(0.999, 0.03))}
    reports = {}
    for eps in EPS:
        fd = np.stack(fd_all[eps])
        report = reports[eps] = {}
        for name, (a, b) in groups.items():
            f, g = fd[:, a:b].ravel(), an_all[:, a:b].ravel()
            corr = float(np.corrcoef(f, g)[0, 1])
            big = np.abs(g) > 0.05 * np.abs(g).max()
            med = float(np.median(np.abs(f[big] - g[big]) / np.abs(g[big])))
            report[name] = (round(corr, 5), round(med, 4))
        print(f"eps {eps}: finite differences vs analytic (correlation, median rel. error of large entries):",
              report)
    for eps, report in reports.items():
        for name, (corr, med) in report.items():
            c_min, m_max = lim[eps][name]
            assert corr > c_min and (m_max is None or med < m_max), (eps, name, report)


def test_gradient_vs_oracle_crop(mods, orc):
    B, AG = mods
    g_np = scenes.gaussians(2_000_000, seed=21, extent=5.0)
    box = np.all(np.abs(g_np["means"]) < 3.0, axis=1)
    idx = np.sort(np.random.default_rng(8).choice(np.nonzero(box)[0], 2000, replace=False))
    crop = {k: np.ascontiguousarray(v[idx]) for k, v in g_np.items()}
    crop["log_scales"] = crop["log_scales"] + 1.0          # fewer, larger splats cover the view
    cam = _cam()
    n = len(idx)
    err, age = scenes.error_map(W, H, seed=4), scenes.age_map(W, H, seed=4)
    T = ((W + 15) // 16) * ((H + 15) // 16)
    from gpu_util import select_dev, select_host
    sel = select_dev(B, err, age, W, H, T // 5, 84, seed=6)
    sh = select_host(sel)
    raster = AG.SampledRaster(cam, n, sel["active_tiles"], sel["n_active"], sel["tile_rank"], sel["pix_off"],
                              sel["pix_idx"], 84)
    leaf = {k: v.requires_grad_(True) for k, v in _dev(crop).items()}
    rgb = AG.render_sampled(leaf, raster)
    P = rgb.shape[0]
    w = np.random.default_rng(3).normal(0, 1e-3, (P, 3)).astype(np.float32)
    (rgb * torch.from_numpy(w).cuda()).sum().backward()
    got = np.concatenate([leaf["means"].grad.cpu().numpy(), leaf["log_scales"].grad.cpu().numpy(),
                          leaf["quats"].grad.cpu().numpy(), leaf["opacity_logits"].grad.cpu().numpy()[:, None],
                          leaf["sh"].grad.reshape(n, 48).cpu().numpy()], 1)
    c64 = {k: v.astype(np.float64) for k, v in crop.items()}
    pr = orc.project(c64, cam, tile_rank=sh["tile_rank"])
    pix = orc.pixel_coords(sh["active_tiles"], sh["pix_off"], sh["pix_idx"], W)
    ref_rgb = orc.render_pixels(pr, W, H, pix)
    ok_pix = ref_rgb["margin"] > 1e-4
    assert ok_pix.mean() > 0.98
    np.testing.assert_array_less(np.abs(rgb.detach().cpu().numpy() - ref_rgb["rgb"])[ok_pix], 1e-4)
    g2 = orc.render_backward(pr, W, H, pix, w.astype(np.float64))
    want = orc.project_backward(c64, cam, g2, tile_rank=sh["tile_rank"])
    ok = pr["margin"] > 1e-4
    assert (np.abs(want[ok]).sum(1) > 0).sum() > 200
    for name, (a, b) in dict(means=(0, 3), scales=(3, 6), quats=(6, 10), opacity=(10, 11), sh_dc=(11, 14),
                             sh_rest=(14, 59)).items():
        r = np.linalg.norm(got[ok, a:b] - want[ok, a:b]) / np.linalg.norm(want[ok, a:b])
        assert r <= 1e-3, (name, r)

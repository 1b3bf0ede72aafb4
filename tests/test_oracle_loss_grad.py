"""Pins of the oracle's sparse loss (Sec. 3.7, App. A) and of its analytic
gradients: NCC invariances, exact zero-sum / scale-orthogonality of the NCC
gradient, the Charbonnier limit, the printed NCC gradient as the epsilon -> 0
limit, EMA/age recurrences, and central finite differences of the loss and of
the whole project -> render -> loss chain."""
import math

import numpy as np
import pytest

from paper_2606_15924_gb300 import scenes


def _tile_sel(W, H, tiles, n_per_tile, rng):
    off, idx = [0], []
    tx_n = (W + 15) // 16
    for t in tiles:
        tx, ty = t % tx_n, t // tx_n
        valid = [l for l in range(256) if 16 * tx + l % 16 < W and 16 * ty + l // 16 < H]
        k = min(n_per_tile, len(valid))
        idx += sorted(rng.choice(valid, k, replace=False).tolist())
        off.append(off[-1] + k)
    return dict(active_tiles=np.array(tiles, np.int32), pix_off=np.array(off, np.int32),
                pix_idx=np.array(idx, np.uint8))


def _gather(target, sel, W):
    import oracle
    P = oracle.pixel_coords(sel["active_tiles"], sel["pix_off"], sel["pix_idx"], W)
    return target[P[:, 1], P[:, 0]]


def test_ncc_invariances(orc):
    W = H = 32
    rng = np.random.default_rng(0)
    target = rng.uniform(0, 1, (H, W, 3))
    sel = _tile_sel(W, H, [0, 3], 40, rng)
    y = _gather(target, sel, W)
    # x = y: NCC = 1 (up to eps), so the loss is the Charbonnier floor
    o = orc.loss(W, H, sel, y, target)
    P = len(y)
    assert o["loss"] == pytest.approx(3 * 1e-3, rel=1e-4)
    # affine: x = 2 y + 0.3 keeps NCC = 1; x = -y gives NCC = -1 -> S-NCC = 2
    lam = np.ones(2)
    o1 = orc.loss(W, H, sel, 2 * y + 0.3, target, lambda_in=lam)
    l1 = np.sqrt((y + 0.3) ** 2 + 1e-6).sum() / P
    assert o1["loss"] - l1 == pytest.approx(0.0, abs=1e-6)
    o2 = orc.loss(W, H, sel, -y, target, lambda_in=lam)
    l2 = np.sqrt((2 * y) ** 2 + 1e-6).sum() / P
    assert o2["loss"] - l2 == pytest.approx(2.0, abs=1e-6)


def test_ncc_gradient_identities(orc):
    """With lambda = 1 and l1 removed (difference of two evaluations), the
    NCC part of dL/dx sums to zero over a tile and is orthogonal to x - mean."""
    W = H = 16
    rng = np.random.default_rng(1)
    target = rng.uniform(0, 1, (H, W, 3))
    sel = _tile_sel(W, H, [0], 60, rng)
    x = rng.uniform(0, 1, (60, 3))
    lam1 = orc.loss(W, H, sel, x, target, lambda_in=np.ones(1))
    lam0 = orc.loss(W, H, sel, x, target, lambda_in=np.zeros(1))
    g = lam1["dL_drgb"] - lam0["dL_drgb"]
    np.testing.assert_allclose(g.sum(0), 0.0, atol=1e-15)
    # sum (x - mx) dNCC/dx = NCC eps / (vx vy + eps): zero as eps -> 0
    y = _gather(target, sel, W)
    mx, my = x.mean(0), y.mean(0)
    vx, vy = ((x - mx) ** 2).mean(0), ((y - my) ** 2).mean(0)
    ncc = ((x - mx) * (y - my)).mean(0) / np.sqrt(vx * vy + 1e-8)
    np.testing.assert_allclose((g * (x - mx)).sum(0), -ncc * 1e-8 / (vx * vy + 1e-8) / 3.0, rtol=1e-6,
                               atol=1e-16)
    a = orc.loss(W, H, sel, x, target, lambda_in=np.ones(1), eps_n=1e-16)
    b = orc.loss(W, H, sel, x, target, lambda_in=np.zeros(1), eps_n=1e-16)
    np.testing.assert_allclose(((a["dL_drgb"] - b["dL_drgb"]) * (x - mx)).sum(0), 0.0, atol=1e-14)


def test_printed_ncc_gradient_is_the_limit(orc):
    """App. A prints dl_NCC/dx = -((y - my)/sqrt(vx vy + eps) - NCC (x - mx)/(vx + eps));
    times 1/n (per tile) and 1/3 (channel mean) it is the exact gradient of
    1 - NCC as eps -> 0."""
    W = H = 16
    rng = np.random.default_rng(2)
    target = rng.uniform(0, 1, (H, W, 3))
    sel = _tile_sel(W, H, [0], 50, rng)
    x = rng.uniform(0, 1, (50, 3))
    y = _gather(target, sel, W)
    a = orc.loss(W, H, sel, x, target, lambda_in=np.ones(1), eps_n=1e-14)
    b = orc.loss(W, H, sel, x, target, lambda_in=np.zeros(1), eps_n=1e-14)
    g = a["dL_drgb"] - b["dL_drgb"]
    n = 50
    mx, my = x.mean(0), y.mean(0)
    vx, vy = ((x - mx) ** 2).mean(0), ((y - my) ** 2).mean(0)
    ncc = ((x - mx) * (y - my)).mean(0) / np.sqrt(vx * vy)
    printed = -((y - my) / np.sqrt(vx * vy) - ncc * (x - mx) / vx)
    np.testing.assert_allclose(g, printed / n / 3.0, rtol=1e-6, atol=1e-12)


def test_charbonnier_limit(orc):
    W = H = 16
    rng = np.random.default_rng(3)
    target = rng.uniform(0, 1, (H, W, 3))
    sel = _tile_sel(W, H, [0], 30, rng)
    x = rng.uniform(0, 1, (30, 3))
    y = _gather(target, sel, W)
    o = orc.loss(W, H, sel, x, target, lambda_in=np.zeros(1), eps_c=1e-12)
    np.testing.assert_allclose(o["dL_drgb"] * 30, np.sign(x - y), atol=1e-9)
    assert o["loss"] == pytest.approx(np.abs(x - y).sum() / 30, rel=1e-9)


def test_loss_finite_differences(orc):
    W, H = 40, 24
    rng = np.random.default_rng(4)
    target = rng.uniform(0, 1, (H, W, 3))
    sel = _tile_sel(W, H, [0, 2, 4, 5], 17, rng)
    P = int(sel["pix_off"][-1])
    x = rng.uniform(0, 1, (P, 3))
    base = orc.loss(W, H, sel, x, target)
    lam = base["lam"]
    assert np.all((lam > 0) & (lam <= 1))
    h = 1e-6
    fd = np.zeros_like(x)
    for p in range(P):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[p, c] += h
            xm[p, c] -= h
            fd[p, c] = (orc.loss(W, H, sel, xp, target, lambda_in=lam)["loss"]
                        - orc.loss(W, H, sel, xm, target, lambda_in=lam)["loss"]) / (2 * h)
    np.testing.assert_allclose(base["dL_drgb"], fd, rtol=1e-6, atol=1e-9)


def test_lambda_reading(orc):
    """lambda = clip(mean |dl1/dx|_1 / (mean |n dNCC/dx|_1 + 1e-8), 0, 1) per tile."""
    W = H = 16
    rng = np.random.default_rng(5)
    target = rng.uniform(0, 1, (H, W, 3))
    sel = _tile_sel(W, H, [0], 40, rng)
    x = rng.uniform(0, 1, (40, 3))
    y = _gather(target, sel, W)
    o = orc.loss(W, H, sel, x, target)
    d = x - y
    g1 = np.abs(d / np.sqrt(d * d + 1e-6)).sum(1).mean()
    n = 40
    mx, my = x.mean(0), y.mean(0)
    vx, vy = ((x - mx) ** 2).mean(0), ((y - my) ** 2).mean(0)
    D = np.sqrt(vx * vy + 1e-8)
    ncc = ((x - mx) * (y - my)).mean(0) / D
    gn = np.abs(((y - my) - ncc * vy * (x - mx) / D) / D).sum(1).mean()
    assert o["lam"][0] == pytest.approx(min(1.0, g1 / (gn + 1e-8)), rel=1e-12)
    del n


def test_lambda_is_clipped_at_one(orc):
    """A prediction that is the target plus a constant has NCC = 1 and a
    vanishing NCC gradient, so the gradient ratio is huge: lambda = 1."""
    W = H = 16
    rng = np.random.default_rng(6)
    target = rng.uniform(0, 0.5, (H, W, 3))
    sel = _tile_sel(W, H, [0], 60, rng)
    y = _gather(target, sel, W)
    o = orc.loss(W, H, sel, y + 0.4, target)
    assert o["lam"][0] == 1.0


def test_ema_and_age_recurrences(orc):
    W, H = 48, 32
    rng = np.random.default_rng(6)
    target = rng.uniform(0, 1, (H, W, 3))
    sel = _tile_sel(W, H, [1, 4], 20, rng)
    P = int(sel["pix_off"][-1])
    x = rng.uniform(0, 1, (P, 3))
    err = scenes.error_map(W, H)
    age = scenes.age_map(W, H, max_age=65535)
    age[0, :5] = 65535
    o = orc.loss(W, H, sel, x, target, err_f16_bits=err, age=age)
    pix = orc.pixel_coords(sel["active_tiles"], sel["pix_off"], sel["pix_idx"], W)
    e = np.abs(x - _gather(target, sel, W)).sum(1)
    np.testing.assert_allclose(o["err"], e, rtol=1e-15)
    want_err = err.copy()
    old = err.view(np.float16).astype(np.float64)[pix[:, 1], pix[:, 0]]
    want_err[pix[:, 1], pix[:, 0]] = (0.6 * old + 0.4 * e).astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(o["err_map"], want_err)
    want_age = np.minimum(age.astype(np.int64) + 1, 65535).astype(np.uint16)
    want_age[pix[:, 1], pix[:, 0]] = 0
    np.testing.assert_array_equal(o["age_map"], want_age)


def test_degenerate_tile(orc):
    W = H = 16
    target = np.full((H, W, 3), 0.25)
    sel = dict(active_tiles=np.array([0], np.int32), pix_off=np.array([0, 1], np.int32),
               pix_idx=np.array([5], np.uint8))
    o = orc.loss(W, H, sel, np.array([[0.5, 0.5, 0.5]]), target)
    assert np.all(np.isfinite(o["dL_drgb"])) and np.isfinite(o["loss"])
    # a single pixel has zero variance: NCC = 0, so S-NCC = 1
    assert o["loss"] == pytest.approx(3 * math.sqrt(0.0625 + 1e-6) + o["lam"][0] * 1.0, rel=1e-12)


# ---------------------------------------------------------------------------
# finite differences of the whole chain
# ---------------------------------------------------------------------------

def _chain_setup(seed=0, n=20):
    W, H = 48, 40
    g = scenes.gaussians(n, seed=seed, log_scale_mean=-0.8, log_scale_std=0.3, sh_std=0.3)
    g = {k: v.astype(np.float64) for k, v in g.items()}
    g["means"] *= 0.6
    cam = scenes.look_at((0.4, -0.3, -4.0), width=W, height=H)
    rng = np.random.default_rng(seed + 50)
    sel = _tile_sel(W, H, [0, 1, 3, 4, 6, 7, 8], 40, rng)
    target = scenes.smooth_image(W, H, seed=seed + 3).astype(np.float64)
    return g, cam, sel, target


def _pack(g):
    n = g["means"].shape[0]
    return np.concatenate([g["means"], g["log_scales"], g["quats"], g["opacity_logits"][:, None],
                           g["sh"].reshape(n, 48)], 1)


def _unpack(p):
    n = p.shape[0]
    return dict(means=p[:, 0:3], log_scales=p[:, 3:6], quats=p[:, 6:10], opacity_logits=p[:, 10],
                sh=p[:, 11:59].reshape(n, 16, 3))


def _forward(orc, p, cam, sel, target, lam=None):
    W, H = cam["width"], cam["height"]
    pr = orc.project(_unpack(p), cam)
    pix = orc.pixel_coords(sel["active_tiles"], sel["pix_off"], sel["pix_idx"], W)
    r = orc.render_pixels(pr, W, H, pix)
    lo = orc.loss(W, H, sel, r["rgb"], target, lambda_in=lam)
    sig = (tuple(pr["radius"]), tuple(r["n_last"]), tuple(r["n_contrib"]),
           tuple((pr["rgb"] > 0).ravel()))
    return lo, r, pr, pix, sig


@pytest.mark.parametrize("seed", [0, 1])
def test_chain_finite_differences(orc, seed):
    g, cam, sel, target = _chain_setup(seed)
    W, H = cam["width"], cam["height"]
    p0 = _pack(g)
    lo, r, pr, pix, sig0 = _forward(orc, p0, cam, sel, target)
    assert (r["n_contrib"] > 0).mean() > 0.6
    lam = lo["lam"]
    g2 = orc.render_backward(pr, W, H, pix, lo["dL_drgb"])
    grads = orc.project_backward(_unpack(p0), cam, g2)
    h = 1e-6
    checked, bad = 0, []
    for i in range(p0.shape[0]):
        for k in range(59):
            pp, pm = p0.copy(), p0.copy()
            pp[i, k] += h
            pm[i, k] -= h
            lp, rp, _, _, sp = _forward(orc, pp, cam, sel, target, lam)
            lm, rm, _, _, sm = _forward(orc, pm, cam, sel, target, lam)
            if sp != sig0 or sm != sig0 or min(rp["margin"].min(), rm["margin"].min()) < 1e-4:
                continue                    # a discrete decision flips inside the stencil
            fd = (lp["loss"] - lm["loss"]) / (2 * h)
            checked += 1
            if abs(fd - grads[i, k]) > 1e-5 * max(abs(fd), 1e-3):
                bad.append((i, k, fd, grads[i, k]))
    assert checked > 0.7 * p0.size, checked
    assert not bad, bad[:10]


def test_chain_finite_differences_clamped_jacobian(orc):
    """The chain's finite differences for large Gaussians whose centres lie
    beyond the Jacobian clamp (x/z or y/z past 1.3 tan of the half field of
    view, on all four sides) while their splats still reach into the image,
    next to two on screen."""
    W, H = 48, 40
    cam = scenes.look_at((0.0, 0.0, -4.0), width=W, height=H)
    d = 4.0
    tx, ty = 0.5 * W / cam["fx"], 0.5 * H / cam["fy"]
    means = np.array([[1.2 * 1.3 * tx * d, 0.1, 0.0], [-1.2 * 1.3 * tx * d, -0.2, 0.3],
                      [0.15, 1.2 * 1.3 * ty * d, 0.0], [-0.1, -1.2 * 1.3 * ty * d, -0.2],
                      [0.2, 0.1, 0.5], [-0.3, -0.2, -0.4]])
    n = len(means)
    rng = np.random.default_rng(8)
    g = dict(means=means, log_scales=np.log(np.array([[0.6, 0.5, 0.7]] * 4 + [[0.2, 0.15, 0.25]] * 2))
             + rng.normal(0.0, 0.05, (n, 3)),
             quats=rng.normal(size=(n, 4)), opacity_logits=rng.normal(0.5, 0.3, n),
             sh=rng.normal(0.0, 0.3, (n, 16, 3)))
    sel = _tile_sel(W, H, list(range(9)), 48, rng)
    target = scenes.smooth_image(W, H, seed=9).astype(np.float64)
    p0 = _pack(g)
    lo, r, pr, pix, sig0 = _forward(orc, p0, cam, sel, target)
    xz = p0[:4, 0] / (p0[:4, 2] + d)
    yz = p0[:4, 1] / (p0[:4, 2] + d)
    assert np.all((np.abs(xz) > 1.3 * tx) | (np.abs(yz) > 1.3 * ty))
    assert np.all(pr["radius"][:4] > 0)                  # clamped, and still reaching the image
    lam = lo["lam"]
    g2 = orc.render_backward(pr, W, H, pix, lo["dL_drgb"])
    grads = orc.project_backward(_unpack(p0), cam, g2)
    h = 1e-6
    checked, bad = 0, []
    for i in range(4):
        for k in range(11):                              # means, scales, rotation, opacity
            pp, pm = p0.copy(), p0.copy()
            pp[i, k] += h
            pm[i, k] -= h
            lp, rp, _, _, sp = _forward(orc, pp, cam, sel, target, lam)
            lm, rm, _, _, sm = _forward(orc, pm, cam, sel, target, lam)
            if sp != sig0 or sm != sig0 or min(rp["margin"].min(), rm["margin"].min()) < 1e-4:
                continue
            fd = (lp["loss"] - lm["loss"]) / (2 * h)
            checked += 1
            if abs(fd - grads[i, k]) > 1e-5 * max(abs(fd), 1e-3):
                bad.append((i, k, fd, grads[i, k]))
    assert checked > 0.7 * 44, checked
    assert not bad, bad[:10]

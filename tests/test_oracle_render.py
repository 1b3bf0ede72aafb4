"""Pins of the oracle's projection, binning and compositing: a closed-form
image of one isotropic Gaussian, the transmittance identity, pixel
independence, and a geometric brute force for tile overlaps."""
import math

import numpy as np
import pytest

from paper_2606_15924_gb300 import scenes


def _one_gaussian(sigma, opacity, dc, d=4.0, W=64, H=48):
    g = dict(means=np.zeros((1, 3)), log_scales=np.full((1, 3), math.log(sigma)),
             quats=np.array([[1.0, 0, 0, 0]]), opacity_logits=np.array([math.log(opacity / (1 - opacity))]),
             sh=np.zeros((1, 16, 3)))
    g["sh"][0, 0, :] = dc
    cam = scenes.look_at((0.0, 0.0, -d), width=W, height=H, fov_x_deg=50.0)
    return g, cam


@pytest.mark.parametrize("sigma,opacity", [(0.05, 0.7), (0.2, 0.3), (0.01, 0.95), (0.4, 0.999)])
def test_closed_form_isotropic_gaussian(orc, sigma, opacity):
    """(0.4, 0.999): alpha near the centre exceeds 0.99 and takes the cap."""
    dc = np.array([0.3, -0.2, 1.1])
    d = 4.0
    g, cam = _one_gaussian(sigma, opacity, dc, d)
    W, H = cam["width"], cam["height"]
    f = cam["fx"]
    # camera on the axis, W = I: Sigma2 = ((f sigma / d)^2 + 0.3) I exactly
    s2 = (f * sigma / d) ** 2 + 0.3
    pr = orc.project(g, cam)
    assert pr["radius"][0] == math.ceil(3.0 * math.sqrt(s2 + math.sqrt(0.1)))
    np.testing.assert_allclose(pr["conic"][0], [1 / s2, 0.0, 1 / s2], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(pr["xy"][0], [W / 2, H / 2], atol=1e-12)
    assert pr["depth"][0] == pytest.approx(d)
    c00 = 0.5 / math.sqrt(math.pi)
    col = np.maximum(0.0, c00 * dc + 0.5)
    ys, xs = np.mgrid[0:H, 0:W]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    out = orc.render_pixels(pr, W, H, pix)
    r2 = (pix[:, 0] + 0.5 - W / 2) ** 2 + (pix[:, 1] + 0.5 - H / 2) ** 2
    alpha = np.minimum(0.99, opacity * np.exp(-r2 / (2 * s2)))
    alpha[alpha < 1 / 255] = 0
    # the splat only reaches tiles its 3-sigma square touches
    rad = pr["radius"][0]
    tx, ty = pix[:, 0] // 16, pix[:, 1] // 16
    inside = ((tx >= math.floor((W / 2 - rad) / 16)) & (tx <= math.floor((W / 2 + rad) / 16))
              & (ty >= math.floor((H / 2 - rad) / 16)) & (ty <= math.floor((H / 2 + rad) / 16)))
    alpha[~inside] = 0
    np.testing.assert_allclose(out["rgb"], alpha[:, None] * col[None, :], atol=1e-12)
    np.testing.assert_allclose(out["T"], 1 - alpha, atol=1e-12)
    if opacity * math.exp(-0.25 / s2) > 0.99:
        assert out["T"].min() == pytest.approx(0.01, abs=1e-15)


def test_transmittance_identity(orc):
    """sum_k T_k alpha_k + T_final = 1: with every colour 1 and black
    background the image is 1 - T_final, with white background it is 1."""
    g = scenes.gaussians(3000, seed=3, log_scale_mean=-2.3)
    cam = scenes.look_at((0, 0, -4), width=64, height=64)
    pr = orc.project(g, cam)
    pr["rgb"] = np.ones_like(pr["rgb"])
    ys, xs = np.mgrid[0:64, 0:64]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    o0 = orc.render_pixels(pr, 64, 64, pix, bg=(0, 0, 0))
    o1 = orc.render_pixels(pr, 64, 64, pix, bg=(1, 1, 1))
    assert (o0["n_contrib"] > 3).mean() > 0.5          # a dense enough scene
    assert (o0["T"] < 2e-3).any()                     # some pixels reach the stop
    np.testing.assert_allclose(o0["rgb"], np.repeat(1 - o0["T"][:, None], 3, 1), atol=1e-12)
    np.testing.assert_allclose(o1["rgb"], 1.0, atol=1e-12)
    # and T_final is the product of (1 - alpha) of the splats blended
    assert np.all(o0["T"] >= 1e-4 - 1e-15) and np.all(o0["T"] <= 1.0)


def test_pixel_independence_and_full_mask(orc):
    g = scenes.gaussians(300, seed=4)
    cam = scenes.look_at((0, 0, -4), width=40, height=36)
    pr = orc.project(g, cam)
    ys, xs = np.mgrid[0:36, 0:40]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    full = orc.render_pixels(pr, 40, 36, pix)
    rng = np.random.default_rng(0)
    sub = rng.choice(len(pix), 200, replace=False)
    part = orc.render_pixels(pr, 40, 36, pix[sub])
    np.testing.assert_array_equal(part["rgb"], full["rgb"][sub])
    np.testing.assert_array_equal(part["T"], full["T"][sub])
    # the full sampling mask lists every valid pixel once, in tile order
    err = scenes.error_map(40, 36)
    age = scenes.age_map(40, 36)
    sel = orc.select(err, age, 40, 36, n_select=10 ** 6, n_pix=256)
    P = orc.pixel_coords(sel["active_tiles"], sel["pix_off"], sel["pix_idx"], 40)
    assert len(P) == 40 * 36
    assert len({(int(a), int(b)) for a, b in P}) == 40 * 36
    dense = orc.render_pixels(pr, 40, 36, P)
    lin = P[:, 1] * 40 + P[:, 0]
    np.testing.assert_array_equal(dense["rgb"], full["rgb"][lin])


def test_bin_tiles_brute_force(orc):
    W, H = 200, 120
    pr = scenes.projected(500, W, H, seed=9)
    tx_n, ty_n = (W + 15) // 16, (H + 15) // 16
    rng = np.random.default_rng(1)
    for masked in (False, True):
        rank = None
        if masked:
            act = rng.uniform(size=tx_n * ty_n) < 0.3
            rank = np.where(act, np.cumsum(act) - 1, -1).astype(np.int32)
        keys, vals, counts = orc.bin_tiles(pr["xy"], pr["radius"], pr["depth"], W, H, rank)
        # geometric definition: tile k overlaps [x - r, x + r] iff 16k <= x + r and 16k + 16 > x - r
        want = []
        for i in range(len(pr["radius"])):
            r = int(pr["radius"][i])
            if r <= 0:
                continue
            x, y = float(pr["xy"][i, 0]), float(pr["xy"][i, 1])
            for ty in range(ty_n):
                if not (16 * ty <= y + r and 16 * ty + 16 > y - r):
                    continue
                for tx in range(tx_n):
                    if not (16 * tx <= x + r and 16 * tx + 16 > x - r):
                        continue
                    t = ty * tx_n + tx
                    if rank is not None and rank[t] < 0:
                        continue
                    want.append((t, float(pr["depth"][i]), i))
        want.sort()
        assert len(want) == len(keys)
        assert [int(v) for v in vals] == [w[2] for w in want]
        assert [int(k >> np.uint64(32)) for k in keys] == [w[0] for w in want]
        dbits = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
        np.testing.assert_array_equal(dbits, pr["depth"][vals])
        assert counts.sum() == len(keys)
        np.testing.assert_array_equal(np.bincount(keys >> np.uint64(32), minlength=tx_n * ty_n).astype(np.int32),
                                      counts)
    # capacity too small is reported
    assert orc.bin_tiles(pr["xy"], pr["radius"], pr["depth"], W, H, None, capacity=3) is None


def test_projection_culls(orc):
    g = scenes.gaussians(50, seed=11)
    g["means"][:10, 2] = -4.1     # behind the camera at z = -4 looking at +z
    g["means"][10:12] = [[0.0, 0.0, -3.85], [0.01, 0.0, -3.75]]   # depth 0.15 < znear = 0.2 < 0.25
    cam = scenes.look_at((0, 0, -4), width=64, height=64)
    pr = orc.project(g, cam)
    assert np.all(pr["radius"][:11] == 0)
    assert pr["radius"][11] > 0
    # an active-tile mask culls splats that touch no active tile
    rank = np.full(16, -1, np.int32)
    pr2 = orc.project(g, cam, tile_rank=rank)
    assert np.all(pr2["radius"] == 0)


def test_error_stats_identities(orc):
    """Sec. 3.8 statistics: the compositing weights of a pixel sum to
    1 - T_final, so sum_i W_i = sum_p (1 - T_final(p)) and sum_i E_i =
    sum_p e(p) (1 - T_final(p)); D is non-negative."""
    g = scenes.gaussians(3000, seed=3, log_scale_mean=-2.3)
    cam = scenes.look_at((0, 0, -4), width=64, height=64)
    pr = orc.project(g, cam)
    ys, xs = np.mgrid[0:64, 0:64]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    rng = np.random.default_rng(5)
    pix = pix[rng.choice(len(pix), 900, replace=False)]
    e = rng.uniform(0.0, 2.0, len(pix))
    st = orc.error_stats(pr, 64, 64, pix, e)
    out = orc.render_pixels(pr, 64, 64, pix)
    assert (out["n_contrib"] > 3).mean() > 0.5
    assert st[:, 1].sum() == pytest.approx((1.0 - out["T"]).sum(), rel=1e-12)
    assert st[:, 0].sum() == pytest.approx((e * (1.0 - out["T"])).sum(), rel=1e-12)
    assert np.all(st[:, 2] >= 0.0) and st[:, 2].sum() > 0.0
    assert np.all(st[pr["radius"] <= 0] == 0.0)


@pytest.mark.parametrize("sigma,opacity", [(0.05, 0.7), (0.2, 0.3)])
def test_error_stats_one_gaussian_closed_form(orc, sigma, opacity):
    """One isotropic Gaussian in front of the camera: T = 1 at every pixel, so
    w = alpha = o exp(-r^2 / (2 s2)) and D = r / sqrt(s2) (s2 the screen-space
    variance), for every pixel whose alpha passes 1/255."""
    dc = np.array([0.3, -0.2, 1.1])
    d = 4.0
    g, cam = _one_gaussian(sigma, opacity, dc, d)
    W, H = cam["width"], cam["height"]
    s2 = (cam["fx"] * sigma / d) ** 2 + 0.3
    pr = orc.project(g, cam)
    ys, xs = np.mgrid[0:H, 0:W]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    e = np.linspace(0.1, 1.0, len(pix))
    st = orc.error_stats(pr, W, H, pix, e)
    r2 = (pix[:, 0] + 0.5 - W / 2) ** 2 + (pix[:, 1] + 0.5 - H / 2) ** 2
    a = np.minimum(0.99, opacity * np.exp(-0.5 * r2 / s2))
    on = a >= 1.0 / 255.0
    # the tile rectangle of the radius bounds which pixels can see the splat
    r = int(pr["radius"][0])
    tx0, tx1 = max(0, int((W / 2 - r) // 16)), min(W // 16, int((W / 2 + r) // 16) + 1)
    ty0, ty1 = max(0, int((H / 2 - r) // 16)), min(H // 16, int((H / 2 + r) // 16) + 1)
    inside = (pix[:, 0] // 16 >= tx0) & (pix[:, 0] // 16 < tx1) & (pix[:, 1] // 16 >= ty0) & (pix[:, 1] // 16 < ty1)
    on &= inside
    assert on.sum() > 20
    assert st[0, 1] == pytest.approx(a[on].sum(), rel=1e-10)
    assert st[0, 0] == pytest.approx((e * a)[on].sum(), rel=1e-10)
    assert st[0, 2] == pytest.approx((np.sqrt(r2 / s2) * a)[on].sum(), rel=1e-10)


@pytest.mark.parametrize("opacity,blended", [(0.6, 10), (0.3, 25), (0.85, 4)])
def test_stop_before_transmittance_falls_below_1e_4(orc, opacity, blended):
    """Co-centred splats along the optical axis, seen at the pixel under
    their common centre (odd image size: the centre is a pixel centre, so
    alpha = opacity exactly): the walk blends k splats while
    (1 - opacity)^k >= 1e-4 and stops before the one that would go below."""
    W, H, n = 65, 49, 40
    k = 0
    while (1.0 - opacity) ** (k + 1) >= 1e-4:
        k += 1
    assert k == blended
    g = dict(means=np.stack([np.zeros(n), np.zeros(n), np.linspace(-1.0, 2.0, n)], 1),
             log_scales=np.full((n, 3), math.log(0.05)), quats=np.tile([1.0, 0, 0, 0], (n, 1)),
             opacity_logits=np.full(n, math.log(opacity / (1 - opacity))), sh=np.zeros((n, 16, 3)))
    g["sh"][:, 0, :] = 0.4
    cam = scenes.look_at((0.0, 0.0, -4.0), width=W, height=H, fov_x_deg=50.0)
    pr = orc.project(g, cam)
    out = orc.render_pixels(pr, W, H, np.array([[32, 24]], np.int32))
    assert out["n_contrib"][0] == blended
    assert out["T"][0] == pytest.approx((1.0 - opacity) ** blended, rel=1e-12)
    col = 0.4 * 0.5 / math.sqrt(math.pi) + 0.5
    assert out["rgb"][0, 0] == pytest.approx(col * (1.0 - (1.0 - opacity) ** blended), rel=1e-12)


@pytest.mark.parametrize("theta", [0.5, -1.2])
def test_error_stats_distance_of_a_rotated_gaussian(orc, theta):
    """Sec. 3.8's distance D = sqrt(d^T Sigma2^-1 d) with its cross term, for a
    rotated anisotropic Gaussian alone (T = 1, w = alpha): Sigma2 from the
    closed form (f / z)^2 Rz D Rz^T + 0.3 I at the image centre; pixels within
    the splat's radius square (inside its tile rectangle)."""
    d, W, H = 4.0, 64, 48
    sc = np.array([0.12, 0.04, 0.05])
    g = dict(means=np.zeros((1, 3)), log_scales=np.log(sc)[None], quats=np.array([[math.cos(theta / 2), 0, 0,
                                                                                     math.sin(theta / 2)]]),
             opacity_logits=np.array([math.log(0.8 / 0.2)]), sh=np.zeros((1, 16, 3)))
    cam = scenes.look_at((0.0, 0.0, -d), width=W, height=H, fov_x_deg=50.0)
    f = cam["fx"]
    c, s_ = math.cos(theta), math.sin(theta)
    Rz = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
    S2 = (f / d) ** 2 * (Rz @ np.diag(sc ** 2) @ Rz.T)[:2, :2] + 0.3 * np.eye(2)
    Q = np.linalg.inv(S2)
    pr = orc.project(g, cam)
    r = int(pr["radius"][0])
    ys, xs = np.mgrid[0:H, 0:W]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    dv = pix + 0.5 - np.array([W / 2, H / 2])
    pix, dv = pix[np.abs(dv).max(1) < r], dv[np.abs(dv).max(1) < r]
    e = np.linspace(0.2, 1.0, len(pix))
    st = orc.error_stats(pr, W, H, pix, e)
    q = np.einsum("pi,ij,pj->p", dv, Q, dv)
    a = np.minimum(0.99, 0.8 * np.exp(-0.5 * q))
    on = a >= 1.0 / 255.0
    assert on.sum() > 50 and abs(Q[0, 1]) > 1e-3 * Q[0, 0]
    assert st[0, 1] == pytest.approx(a[on].sum(), rel=1e-9)
    assert st[0, 2] == pytest.approx((np.sqrt(q) * a)[on].sum(), rel=1e-9)


def test_jacobian_clamp_off_screen(orc):
    """A large isotropic Gaussian beyond the right edge, at x/z = 1.5
    tan(fov_x / 2) (outside the 1.3 clamp), still reaching into the image:
    its centre uses the true x/z, its covariance J with x/z clamped to
    1.3 tan(fov_x / 2): Sigma2 = s^2 J J^T + 0.3 I."""
    d, W, H, s = 4.0, 64, 48, 0.5
    cam = scenes.look_at((0.0, 0.0, -d), width=W, height=H, fov_x_deg=50.0)
    f = cam["fx"]
    half = 0.5 * W / f
    x0 = 1.5 * half * d
    g = dict(means=np.array([[x0, 0.0, 0.0]]), log_scales=np.full((1, 3), math.log(s)),
             quats=np.array([[1.0, 0, 0, 0]]), opacity_logits=np.array([2.0]), sh=np.zeros((1, 16, 3)))
    pr = orc.project(g, cam)
    assert pr["radius"][0] > 0
    np.testing.assert_allclose(pr["xy"][0], [f * x0 / d + W / 2, H / 2], rtol=1e-12)
    tx = 1.3 * half
    J = np.array([[f / d, 0.0, -f * tx / d], [0.0, f / d, 0.0]])
    S2 = s * s * J @ J.T + 0.3 * np.eye(2)
    inv = np.linalg.inv(S2)
    np.testing.assert_allclose(pr["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-10)

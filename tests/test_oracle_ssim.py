"""Pins of the oracle's sparse loss with the SSIM structure term (the S-SSIM
variant of Table 4; SSIM after Wang et al. 2004 with C1 = 0.01^2 and
C2 = 0.03^2, per colour channel over a tile's sampled pixels):

- a prediction equal to the target scores SSIM = 1 in every tile, leaving
  only the Charbonnier floor, and its structure gradient is zero;
- the loss is symmetric in prediction and target (with the weight fixed);
- central finite differences of the loss match dL/dI;
- the structure part lies in [0, 2] (|SSIM| <= 1);
- constant tiles reduce SSIM to its luminance factor
  (2 a b + C1) / (a^2 + b^2 + C1), a textbook special case that pins C1;
- a prediction mirrored about the target's mean (x = 2 m - y) keeps the
  luminance factor at 1 and leaves the contrast-structure factor
  (C2 - 2 var) / (2 var + C2), which pins C2 and the sign of the covariance;
- the error and age maps follow Eqs. 3-4 exactly as with the NCC term."""
import numpy as np
import pytest

from paper_2606_15924_gb300 import scenes

W = H = 64
C1, C2 = 0.01 ** 2, 0.03 ** 2


def _sel(orc, n_select=8, n_pix=40, seed=3):
    err, age = scenes.error_map(W, H, seed=seed), scenes.age_map(W, H, seed=seed)
    return orc.select(err, age, W, H, n_select=n_select, n_pix=n_pix, seed=seed), err, age


def _pix(orc, sel):
    return orc.pixel_coords(sel["active_tiles"], sel["pix_off"], sel["pix_idx"], W)


def test_equal_images_score_one(orc):
    sel, err, age = _sel(orc)
    tgt = scenes.smooth_image(W, H, seed=5).astype(np.float64)
    pix = _pix(orc, sel)
    rgb = tgt[pix[:, 1], pix[:, 0]]
    out = orc.loss_ssim(W, H, sel, rgb, tgt)
    assert out["loss"] == pytest.approx(3 * 1e-3, rel=1e-12)       # sum_c sqrt(0 + eps_c^2) per pixel
    assert np.all(out["dL_drgb"] == 0.0)


def test_symmetric_in_prediction_and_target(orc):
    sel, _, _ = _sel(orc)
    rng = np.random.default_rng(1)
    pix = _pix(orc, sel)
    tgt = rng.uniform(0, 1, (H, W, 3))
    rgb = rng.uniform(0, 1, (len(pix), 3))
    A = sel["n_active"]
    lam = np.ones(A)
    a = orc.loss_ssim(W, H, sel, rgb, tgt, lambda_in=lam)["loss"]
    tgt2 = np.zeros((H, W, 3))
    tgt2[pix[:, 1], pix[:, 0]] = rgb
    b = orc.loss_ssim(W, H, sel, tgt[pix[:, 1], pix[:, 0]], tgt2, lambda_in=lam)["loss"]
    assert a == pytest.approx(b, rel=1e-12)


def test_finite_differences(orc):
    sel, _, _ = _sel(orc, n_select=4, n_pix=30)
    rng = np.random.default_rng(2)
    pix = _pix(orc, sel)
    tgt = rng.uniform(0, 1, (H, W, 3))
    rgb = np.clip(tgt[pix[:, 1], pix[:, 0]] + rng.normal(0, 0.2, (len(pix), 3)), 0, 1)
    base = orc.loss_ssim(W, H, sel, rgb, tgt)
    lam = base["lam"]
    g = base["dL_drgb"]
    eps = 1e-6
    for k in rng.choice(len(pix) * 3, 40, replace=False):
        r1, r2 = rgb.copy().reshape(-1), rgb.copy().reshape(-1)
        r1[k] += eps
        r2[k] -= eps
        l1 = orc.loss_ssim(W, H, sel, r1.reshape(-1, 3), tgt, lambda_in=lam)["loss"]
        l2 = orc.loss_ssim(W, H, sel, r2.reshape(-1, 3), tgt, lambda_in=lam)["loss"]
        fd = (l1 - l2) / (2 * eps)
        assert fd == pytest.approx(g.reshape(-1)[k], rel=1e-5, abs=1e-10)


def test_structure_part_within_bounds(orc):
    rng = np.random.default_rng(3)
    for seed in range(5):
        sel, _, _ = _sel(orc, seed=seed)
        pix = _pix(orc, sel)
        tgt = rng.uniform(0, 1, (H, W, 3))
        rgb = rng.uniform(0, 1, (len(pix), 3))
        A = sel["n_active"]
        out = orc.loss_ssim(W, H, sel, rgb, tgt, lambda_in=np.ones(A), eps_c=0.0)
        structure = out["loss"] - out["err"].sum() / len(pix)    # with eps_c = 0, l1 = e
        assert 0.0 <= structure <= 2.0


def _one_tile(orc, n_pix):
    sel = orc.select(np.zeros((H, W), np.uint16), np.zeros((H, W), np.uint16), W, H, n_select=1, n_pix=n_pix)
    return sel, _pix(orc, sel)


def test_constant_tiles_reduce_to_luminance(orc):
    sel, pix = _one_tile(orc, 50)
    a, b = np.array([0.2, 0.5, 0.9]), np.array([0.6, 0.5, 0.1])
    tgt = np.zeros((H, W, 3))
    tgt[pix[:, 1], pix[:, 0]] = b
    rgb = np.tile(a, (len(pix), 1))
    out = orc.loss_ssim(W, H, sel, rgb, tgt, lambda_in=np.ones(1), eps_c=0.0)
    lum = (2 * a * b + C1) / (a * a + b * b + C1)
    structure = out["loss"] - out["err"].sum() / len(pix)
    assert structure == pytest.approx(1.0 - lum.mean(), rel=1e-12)


def test_mirrored_prediction_pins_contrast_structure(orc):
    sel, pix = _one_tile(orc, 64)
    rng = np.random.default_rng(6)
    y = rng.uniform(0.2, 0.8, (len(pix), 3))
    tgt = np.zeros((H, W, 3))
    tgt[pix[:, 1], pix[:, 0]] = y
    m = y.mean(0)
    x = 2 * m - y                                   # same mean, covariance -var
    out = orc.loss_ssim(W, H, sel, x, tgt, lambda_in=np.ones(1), eps_c=0.0)
    var = ((y - m) ** 2).mean(0)
    cs = (C2 - 2 * var) / (2 * var + C2)
    structure = out["loss"] - out["err"].sum() / len(pix)
    assert structure == pytest.approx(1.0 - cs.mean(), rel=1e-10)


def test_maps_as_with_ncc(orc):
    sel, err, age = _sel(orc)
    rng = np.random.default_rng(7)
    pix = _pix(orc, sel)
    tgt = rng.uniform(0, 1, (H, W, 3))
    rgb = rng.uniform(0, 1, (len(pix), 3))
    a = orc.loss_ssim(W, H, sel, rgb, tgt, err_f16_bits=err, age=age)
    b = orc.loss(W, H, sel, rgb, tgt, err_f16_bits=err, age=age)
    np.testing.assert_array_equal(a["err_map"], b["err_map"])
    np.testing.assert_array_equal(a["age_map"], b["age_map"])
    np.testing.assert_array_equal(a["err"], b["err"])

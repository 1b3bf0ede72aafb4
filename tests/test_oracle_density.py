"""Pins of the oracle's Gaussian difficulty scores (Sec. 3.8, Eq. 13) on top of
the statistics of Eq. 12: a constant pixel error gives that error as the
score (a weighted mean), the distance score of one isotropic Gaussian is the
alpha-weighted mean of its closed-form Mahalanobis distances, the scores do
not change when every view is counted twice (the visibility normalisation),
the distance weight fades from lambda_base to 0 with training progress, and
an unseen Gaussian scores 0."""
import math

import numpy as np
import pytest

from paper_2606_15924_gb300 import scenes


def _one_gaussian_stats(orc, err):
    sigma, opacity, d = 0.1, 0.7, 4.0
    g = dict(means=np.zeros((1, 3)), log_scales=np.full((1, 3), math.log(sigma)),
             quats=np.array([[1.0, 0, 0, 0]]), opacity_logits=np.array([math.log(opacity / (1 - opacity))]),
             sh=np.zeros((1, 16, 3)))
    cam = scenes.look_at((0.0, 0.0, -d), width=64, height=48, fov_x_deg=50.0)
    pr = orc.project(g, cam)
    r = int(pr["radius"][0])
    ys, xs = np.mgrid[0:48, 0:64]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    dv = pix + 0.5 - np.array([32.0, 24.0])
    keep = np.abs(dv).max(1) < r                      # inside the splat's tile rectangle
    pix, dv = pix[keep], dv[keep]
    st = orc.error_stats(pr, 64, 48, pix, err(len(pix)))
    s2 = (cam["fx"] * sigma / d) ** 2 + 0.3
    q = (dv ** 2).sum(1) / s2
    a = np.minimum(0.99, opacity * np.exp(-0.5 * q))
    on = a >= 1.0 / 255.0
    return st, a[on], np.sqrt(q[on])


def test_constant_error_scores_that_error(orc):
    st, _, _ = _one_gaussian_stats(orc, lambda n: np.full(n, 0.37))
    # inside Eq. 13's stated range rho in [0, 1): e is the error itself, the
    # distance term only adds to s
    for t in (0, 1000, 3000):
        e, s = orc.gaussian_scores(st, t=t)
        assert e[0] == pytest.approx(0.37, rel=1e-7) and s[0] > e[0]
    # the end point rho = 1 (Alg. 1's min(1, t / tau_until) from tau_until on): no distance term
    e, s = orc.gaussian_scores(st, t=10 ** 6)
    assert e[0] == pytest.approx(0.37, rel=1e-7) and s[0] == pytest.approx(0.37, rel=1e-7)


def test_distance_score_is_the_weighted_mean_distance(orc):
    st, a, D = _one_gaussian_stats(orc, lambda n: np.linspace(0.1, 0.9, n))
    e0, s0 = orc.gaussian_scores(st, t=0)             # lambda_eff = lambda_base = 0.8
    d_mean = (a * D).sum() / a.sum()
    assert s0[0] - e0[0] == pytest.approx(0.8 * d_mean, rel=1e-7)
    # halfway through, half the weight
    e1, s1 = orc.gaussian_scores(st, t=1750)
    assert s1[0] - e1[0] == pytest.approx(0.4 * d_mean, rel=1e-7)
    assert e1[0] == e0[0]


def test_scores_ignore_how_often_a_gaussian_is_seen(orc):
    rng = np.random.default_rng(4)
    st = np.abs(rng.normal(size=(50, 4))) * np.array([2.0, 5.0, 9.0, 0.0])
    st[:, 1] += 0.5                                   # visibilities well above eps = 1e-8
    e1, s1 = orc.gaussian_scores(st, t=300)
    e2, s2 = orc.gaussian_scores(st * 2.0, t=300)     # every view counted twice
    np.testing.assert_allclose(e2, e1, rtol=1e-7)
    np.testing.assert_allclose(s2, s1, rtol=1e-7)
    assert np.all(s1 >= e1)


def test_unseen_gaussians_score_zero(orc):
    st = np.zeros((3, 4))
    st[1] = (0.2, 0.5, 1.5, 0.0)
    e, s = orc.gaussian_scores(st, t=0)
    assert e[0] == s[0] == 0.0 and e[2] == s[2] == 0.0
    assert np.all(np.isfinite(e)) and e[1] > 0.0 and s[1] > e[1]

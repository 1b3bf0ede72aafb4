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


# ---------------------------------------------------------------------------
# densification and pruning (Sec. 3.8 Eq. 13; Alg. 1 step 11; Table 6)
# ---------------------------------------------------------------------------

def _rows(n, seed=0):
    rng = np.random.default_rng(seed)
    p = np.zeros((n, 59), np.float32)
    p[:, 0:3] = rng.uniform(-1, 1, (n, 3))
    p[:, 3:6] = rng.normal(-3.0, 0.5, (n, 3))
    q = rng.normal(size=(n, 4))
    p[:, 6:10] = q / np.linalg.norm(q, axis=1, keepdims=True)
    p[:, 10] = rng.normal(0.0, 1.0, n)
    p[:, 11:] = rng.normal(0.0, 0.2, (n, 48))
    return p


def test_screen_grad_accumulation(orc):
    g = np.zeros((4, 12), np.float32)
    g[0, 0:2] = (3.0, 4.0)                 # |(3, 4)| = 5
    g[2, 5] = 1e-3                         # touched through the opacity only: norm 0, counted
    acc = np.zeros((4, 2), np.float32)
    for _ in range(3):                     # three views
        orc.accumulate_screen_grad(g, acc)
    np.testing.assert_array_equal(acc, [[15.0, 3.0], [0.0, 0.0], [0.0, 3.0], [0.0, 0.0]])


def test_densify_takes_the_top_scored_candidates(orc):
    n = 40
    p = _rows(n)
    p[:, 10] = 2.0                          # nobody pruned
    rng = np.random.default_rng(1)
    st = np.zeros((n, 4), np.float32)
    st[:, 1] = rng.uniform(0.5, 2.0, n)
    st[:, 0] = rng.uniform(0.0, 1.0, n) * st[:, 1]
    st[:, 2] = rng.uniform(0.0, 3.0, n) * st[:, 1]
    st[5, 1] = 0.0                          # unseen: never a candidate
    ac = np.zeros((n, 2), np.float32)
    ac[:, 1] = 2.0
    ac[:, 0] = np.where(np.arange(n) % 3 == 0, 1e-5, 1e-3)   # every third below tau_grad
    ac[7] = ac[11]                          # equal statistics: the tie goes to the lower index
    st[7] = st[11]
    lam = np.float32(0.8 * (1 - 0.25))
    out, src, kind = orc.density_control(p, st, ac, lam, 2e-4, log_split=10.0, logit_prune=-5.3, topk_pm=500)
    # brute force: the candidates and their scores in single precision, sorted by Python
    e = st[:, 0] / (st[:, 1] + np.float32(1e-8))
    d = st[:, 2] / (st[:, 1] + np.float32(1e-8))
    s = e + lam * d
    cand = [i for i in range(n) if st[i, 1] > 0 and ac[i, 0] / max(ac[i, 1], 1) >= np.float32(2e-4)]
    ranked = sorted(cand, key=lambda i: (-float(s[i]), i))
    want = set(ranked[:len(cand) * 500 // 1000])
    got = set(src[kind == 1].tolist())
    assert got == want and len(got) == len(cand) // 2
    assert len(out) == n + len(want)
    assert np.all(np.diff(src) >= 0)                         # input order kept
    for i in want:                                           # clones are exact copies, right after the original
        rows = np.where(src == i)[0]
        assert list(kind[rows]) == [0, 1]
        np.testing.assert_array_equal(out[rows[0]], p[i].astype(np.float64))
        np.testing.assert_array_equal(out[rows[1]], p[i].astype(np.float64))


def test_split_children_along_the_principal_axis(orc):
    Rotation = pytest.importorskip("scipy.spatial.transform").Rotation
    n = 12
    p = _rows(n, seed=3)
    p[:, 10] = 2.0
    st = np.ones((n, 4), np.float32)
    ac = np.tile(np.array([[1.0, 1.0]], np.float32), (n, 1))
    out, src, kind = orc.density_control(p, st, ac, 0.0, 2e-4, log_split=-100.0, logit_prune=-5.3, topk_pm=1000)
    assert len(out) == 2 * n and np.all(kind[0::2] == 2) and np.all(kind[1::2] == 3)
    for i in range(n):
        a, b = out[2 * i], out[2 * i + 1]
        mu = p[i, 0:3].astype(np.float64)
        off = a[0:3] - mu
        np.testing.assert_allclose((a[0:3] + b[0:3]) / 2, mu, atol=1e-12)
        k = int(np.argmax(p[i, 3:6]))
        sig = np.exp(p[i, 3:6].astype(np.float64))
        assert np.linalg.norm(off) == pytest.approx(sig[k], rel=1e-9)
        # the offset is the eigenvector of Sigma = R S^2 R^T with the largest eigenvalue
        w, x, y, z = p[i, 6:10].astype(np.float64)
        R = Rotation.from_quat([x, y, z, w]).as_matrix()
        Sig = R @ np.diag(sig ** 2) @ R.T
        np.testing.assert_allclose(Sig @ off, sig[k] ** 2 * off, rtol=1e-9, atol=1e-15)
        np.testing.assert_allclose(a[3:6], p[i, 3:6] - np.log(1.6), atol=1e-6)
        np.testing.assert_array_equal(a[6:], p[i, 6:].astype(np.float64))


def test_pruning(orc):
    n = 30
    p = _rows(n, seed=4)
    p[:, 10] = np.where(np.arange(n) % 4 == 0, -6.0, 1.0)    # opacity 0.0025 < 0.005 every fourth
    rng = np.random.default_rng(5)
    st = np.zeros((n, 4), np.float32)
    st[:, 1] = rng.uniform(0.0, 1.0, n)
    ac = np.zeros((n, 2), np.float32)
    lp = np.float32(np.log(0.005 / 0.995))
    out, src, kind = orc.density_control(p, st, ac, 0.5, 2e-4, 10.0, lp)
    assert set(src.tolist()) == {i for i in range(n) if i % 4} and np.all(kind == 0)
    # final pruning: also everything outside the 60 % with the largest W
    out, src, kind = orc.density_control(p, st, ac, 0.5, 2e-4, 10.0, lp, final=True, final_pm=600)
    top = sorted(range(n), key=lambda i: (-float(st[i, 1]), i))[:n * 600 // 1000]
    assert set(src.tolist()) == {i for i in top if i % 4}


def test_equal_scores_at_the_cut_go_to_the_lower_index(orc):
    n = 6
    p = _rows(n, seed=6)
    p[:, 10] = 2.0
    st = np.tile(np.array([[0.5, 1.0, 0.2, 0.0]], np.float32), (n, 1))   # every score equal
    ac = np.tile(np.array([[1.0, 1.0]], np.float32), (n, 1))
    out, src, kind = orc.density_control(p, st, ac, 0.5, 2e-4, 10.0, -5.3, topk_pm=500)
    assert sorted(src[kind == 1].tolist()) == [0, 1, 2]

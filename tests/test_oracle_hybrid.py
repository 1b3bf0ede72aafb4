"""Pins of the oracle's hybrid solver (Sec. 3.9, App. A): Cholesky against an
LU solve, J = 0, the rank-1 case against Sherman-Morrison, the diagonal mode
in closed form, and the Adam steps in closed form."""
import numpy as np
import pytest

CFG = np.array([1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3, 0.9, 0.999, 1e-15, 1e-8])


def _lr(k):
    return CFG[0 if k < 3 else 1 if k < 6 else 2 if k < 10 else 3 if k == 10 else 4 if k < 14 else 5]


def test_cholesky_vs_lu(orc):
    rng = np.random.default_rng(0)
    for d in (1, 4, 10, 14):
        M = rng.normal(size=(d, d))
        A = M @ M.T + d * np.eye(d)
        b = rng.normal(size=d)
        np.testing.assert_allclose(orc.cholesky_solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-14)
    with pytest.raises(np.linalg.LinAlgError):
        orc.cholesky_solve(-np.eye(3), np.ones(3))


def _state(n, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=(n, 59))
    g = rng.normal(scale=0.05, size=(n, 59))
    m = rng.normal(scale=0.01, size=(n, 59))
    v = rng.uniform(1e-6, 1e-3, size=(n, 59))
    return p, g, m, v


def test_zero_jacobian_is_moment_ratio(orc):
    """J = 0 (zero view rows): D = -m / (sqrt(v) + eps_lm) on both LM blocks."""
    p, g, m, v = _state(5, 1)
    rows = np.zeros((1, 5, 14))
    pn, mn, vn = orc.hybrid_step(p, g, m, v, np.ones(5), step=3, mode=2, cfg=CFG, rows=rows)
    m1 = 0.9 * m + 0.1 * g
    v1 = 0.999 * v + 0.001 * g * g
    np.testing.assert_allclose(mn, m1, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(vn, v1, rtol=1e-12)
    for k in list(range(10)) + [10, 11, 12, 13]:
        want = p[:, k] + _lr(k) * (-m1[:, k] / (np.sqrt(v1[:, k]) + 1e-8))
        np.testing.assert_allclose(pn[:, k], want, rtol=1e-12)


def test_rank_one_sherman_morrison(orc):
    """Single view row J = g^T: (g g^T + D) x = -m solved in closed form."""
    p, g, m, v = _state(6, 2)
    pn, mn, vn = orc.hybrid_step(p, g, m, v, np.ones(6), step=1, mode=2, cfg=CFG)
    for i in range(6):
        for idx in (list(range(10)), [11, 12, 13, 10]):
            gg = g[i, idx]
            Dg = np.sqrt(vn[i, idx]) + 1e-8
            rhs = -mn[i, idx]
            Dinv_r = rhs / Dg
            Dinv_g = gg / Dg
            x = Dinv_r - Dinv_g * (gg @ Dinv_r) / (1.0 + gg @ Dinv_g)
            lr = np.array([_lr(k) for k in idx])
            np.testing.assert_allclose(pn[i, idx], p[i, idx] + lr * x, rtol=1e-10, atol=1e-15)


def test_multi_row_cholesky_vs_lu(orc):
    p, g, m, v = _state(4, 3)
    rows = np.random.default_rng(9).normal(scale=0.05, size=(3, 4, 14))
    pn, mn, vn = orc.hybrid_step(p, g, m, v, np.ones(4), step=2, mode=2, cfg=CFG, rows=rows)
    for i in range(4):
        for off, idx in ((0, list(range(10))), (10, [11, 12, 13, 10])):
            d = len(idx)
            J = rows[:, i, off:off + d]
            A = J.T @ J + np.diag(np.sqrt(vn[i, idx]) + 1e-8)
            x = np.linalg.solve(A, -mn[i, idx])
            lr = np.array([_lr(k) for k in idx])
            np.testing.assert_allclose(pn[i, idx], p[i, idx] + lr * x, rtol=1e-10, atol=1e-15)


def test_diagonal_mode_closed_form(orc):
    p, g, m, v = _state(7, 4)
    pn, mn, vn = orc.hybrid_step(p, g, m, v, np.ones(7), step=5, mode=1, cfg=CFG)
    for k in list(range(14)):
        want = p[:, k] + _lr(k) * (-mn[:, k] / (g[:, k] ** 2 + np.sqrt(vn[:, k]) + 1e-8))
        np.testing.assert_allclose(pn[:, k], want, rtol=1e-12)


def test_adam_closed_form_and_touched(orc):
    p, g, m, v = _state(8, 5)
    touched = np.array([1, 0, 1, 1, 0, 1, 1, 1], np.uint8)
    m0, v0 = np.zeros_like(m), np.zeros_like(v)
    pn, mn, vn = orc.hybrid_step(p, g, m0, v0, touched, step=1, mode=0, cfg=CFG)
    # first Adam step from zero moments: -lr * g / (|g| + eps)
    t = touched.astype(bool)
    lr = np.array([_lr(k) for k in range(59)])
    np.testing.assert_allclose(pn[t], p[t] - lr * g[t] / (np.abs(g[t]) + 1e-15), rtol=1e-9)
    np.testing.assert_array_equal(pn[~t], p[~t])
    np.testing.assert_array_equal(mn[~t], 0.0)
    # higher SH in LM modes take the bias-corrected Adam step
    pn2, mn2, vn2 = orc.hybrid_step(p, g, m, v, np.ones(8), step=4, mode=1, cfg=CFG)
    mh = mn2[:, 14:] / (1 - 0.9 ** 4)
    vh = vn2[:, 14:] / (1 - 0.999 ** 4)
    np.testing.assert_allclose(pn2[:, 14:], p[:, 14:] - CFG[5] * mh / (np.sqrt(vh) + 1e-15), rtol=1e-12)

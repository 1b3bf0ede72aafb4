"""Pins of the oracle's tile memory, features and error-map refresh (the
tile-error predictor's inputs and its use), against what their definitions
fix: means by grouping, the geometry of the tile ray, invariants of the
rescaling."""
import math

import numpy as np

from paper_2606_15924_gb300 import scenes


def test_observe_means_by_grouping(orc):
    rng = np.random.default_rng(0)
    T, A = 40, 12
    active = np.sort(rng.choice(T, A, replace=False)).astype(np.int32)
    counts = rng.integers(1, 30, A)
    pix_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    P = int(pix_off[-1])
    Tf = rng.uniform(0, 1, P)
    err = rng.exponential(0.2, P)
    ranges = np.stack([np.arange(A) * 100, np.arange(A) * 100 + rng.integers(0, 90, A)], 1).astype(np.int32)
    mem = np.zeros((T, 4))
    mem_it = np.zeros(T, dtype=np.int64)
    tgt = orc.tile_observe(A, active, pix_off, ranges, Tf, err, 77, mem, mem_it)
    owner = np.repeat(np.arange(A), counts)
    mean_e = np.bincount(owner, weights=err) / counts
    mean_t = np.bincount(owner, weights=Tf) / counts
    np.testing.assert_allclose(tgt, np.log1p(mean_e), rtol=1e-12)
    np.testing.assert_allclose(mem[active, 2], mean_e, rtol=1e-12)
    np.testing.assert_allclose(mem[active, 1], mean_t, rtol=1e-12)
    np.testing.assert_array_equal(mem[active, 0], ranges[:, 1] - ranges[:, 0])
    assert np.all(mem[active, 3] == 1) and np.all(mem_it[active] == 77)
    rest = np.setdiff1d(np.arange(T), active)
    assert np.all(mem[rest] == 0) and np.all(mem_it[rest] == 0)


def test_features_ray_geometry_and_unseen_tiles(orc):
    cam = scenes.look_at((0.0, 0.0, -4.0), width=64, height=48)
    cam = dict(cam, cx=24.0, cy=8.0)          # principal point at the centre of tile (1, 0)
    T = 4 * 3
    mem = np.zeros((T, 4))
    mem_it = np.zeros(T, dtype=np.int64)
    mem[5] = [99.0, 0.25, 0.5, 1.0]
    mem_it[5] = 40
    x = orc.tile_features(mem, mem_it, cam, view_cos=0.5, iter_=50)
    assert x[1, 5] == 1.0                       # the ray through the principal point is the axis
    for t in range(T):
        u = ((t % 4) * 16 + 8 - cam["cx"]) / cam["fx"]
        v = ((t // 4) * 16 + 8 - cam["cy"]) / cam["fy"]
        ray = np.array([u, v, 1.0])
        assert math.isclose(x[t, 5], ray[2] / np.linalg.norm(ray), rel_tol=1e-12)
    np.testing.assert_allclose(x[5, :7], [math.log1p(99), 0.25, math.log1p(0.5), 0.5, math.log1p(10), x[5, 5], 1])
    unseen = [t for t in range(T) if t != 5]
    assert np.all(x[unseen, 1] == 1.0) and np.all(x[unseen, 6] == 0.0)
    assert np.allclose(x[unseen, 4], math.log1p(1e6)) and np.all(x[:, 7:] == 0)
    xr = orc.tile_features(mem, mem_it, cam, rows=np.array([5, 0], dtype=np.int32), view_cos=0.5, iter_=50)
    np.testing.assert_array_equal(xr, x[[5, 0]])


def test_refresh_sets_tile_means_and_keeps_shape(orc):
    W, H = 40, 20                                 # ragged tiles at the right and bottom edges
    bits = scenes.error_map(W, H, seed=4)
    bits[0:16, 16:32] = 0                         # one tile of zeros
    tx, ty = 3, 2
    pred = np.random.default_rng(1).uniform(-0.2, 1.5, tx * ty)
    out = orc.tile_refresh(pred, bits, W, H)
    e0 = bits.view(np.float16).astype(np.float64)
    e1 = out.view(np.float16).astype(np.float64)
    for t in range(tx * ty):
        sl = (slice((t // tx) * 16, min(H, (t // tx) * 16 + 16)), slice((t % tx) * 16, min(W, (t % tx) * 16 + 16)))
        want = math.expm1(max(pred[t], 0.0))
        assert abs(e1[sl].mean() - want) <= 2e-3 * max(want, 1e-3) + 1e-7, t
        a, b = e0[sl].ravel(), e1[sl].ravel()
        if a.max() > 0:
            k = a > 1e-3 * a.max()
            r = b[k] / a[k]
            assert np.all(np.abs(r / np.median(r) - 1) < 2e-3), t      # the shape is kept
        else:
            assert np.all(b == e1[sl].ravel()[0]) and abs(b[0] - want) <= 1e-3 * max(want, 1e-3)


def test_residual_targets_and_base(orc):
    T = 6
    mem = np.zeros((T, 4))
    mem_it = np.zeros(T, dtype=np.int64)
    act = np.array([1, 4], dtype=np.int32)
    off = np.array([0, 2, 3], dtype=np.int32)
    rg = np.array([[0, 5], [5, 9]], dtype=np.int32)
    t1 = orc.tile_observe(2, act, off, rg, np.ones(3), np.array([0.2, 0.4, 0.1]), 1, mem, mem_it, residual=True)
    np.testing.assert_allclose(t1, np.log1p([0.3, 0.1]))           # no previous observation: absolute
    t2 = orc.tile_observe(1, act[1:], off[:2], rg[1:], np.ones(2), np.array([0.5, 0.7]), 2, mem, mem_it,
                          residual=True)
    np.testing.assert_allclose(t2, [np.log1p(0.6) - np.log1p(0.1)])
    cam = dict(viewmat=np.eye(4), fx=50.0, fy=50.0, cx=24.0, cy=8.0, width=48, height=32, znear=0.2)
    x = orc.tile_features(mem, mem_it, cam, iter_=3)
    bits = np.full((32, 48), np.float16(0.25)).view(np.uint16)
    out = orc.tile_refresh(np.zeros(T), bits, 48, 32, base=x).view(np.float16).astype(np.float64)
    assert abs(out[0:16, 16:32].mean() - 0.3) < 1e-3                 # tile 1: its last observed error
    assert abs(out[16:32, 16:32].mean() - 0.6) < 1e-3                # tile 4
    assert np.all(out[0:16, 0:16] == 0)                              # never observed, zero residual


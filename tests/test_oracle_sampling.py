"""Pins of the oracle's tile selection and tile-wise pixel sampling (Sec. 3.5):
exact counts, brute-force TopK, the error-proportional draw against exact
enumeration of successive weighted draws without replacement, uniformity of
the remainder, and structural properties of the sampled set."""
import itertools
import math

import numpy as np
import pytest

from paper_2606_15924_gb300 import scenes


def _seq_inclusion(p, k):
    """Exact inclusion probabilities of k successive draws without
    replacement, each proportional to the remaining weights."""
    n = len(p)
    inc = np.zeros(n)
    for order in itertools.permutations(range(n), k):
        pr, rem = 1.0, 1.0
        for i in order:
            pr *= p[i] / rem
            rem -= p[i]
        for i in order:
            inc[i] += pr
    return inc


def test_split_counts_and_extremes(orc):
    w = np.arange(1, 11, dtype=np.uint64) * 1000
    age = np.arange(10, dtype=np.uint32)
    assert orc.choose_items(w, age, 0).sum() == 0
    assert orc.choose_items(w, age, 10).all()
    assert orc.choose_items(w, age, 99).all()
    for n in range(11):
        assert orc.choose_items(w, age, n, seed=3).sum() == n


@pytest.mark.parametrize("hard_pm,stable_pm", [(400, 600), (500, 500), (400, 300)])
def test_split_rounds_half_up_and_clamps(orc, hard_pm, stable_pm):
    """N_hard = round(r_hard n), N_stable = round(r_stable n) (halves up),
    N_stable cut so that N_hard + N_stable <= n.  Items 0..n-1 carry all the
    weight and items n..2n-1 all the age, so the hard draw can only take the
    first group and the oldest-first draw the second."""
    for n in range(1, 13):
        kh = int(math.floor(hard_pm * n / 1000 + 0.5))
        ks = min(int(math.floor(stable_pm * n / 1000 + 0.5)), n - kh)
        w = np.zeros(3 * n, np.uint64)
        w[:n] = 1000
        age = np.zeros(3 * n, np.uint32)
        age[n:2 * n] = 50
        got = orc.choose_items(w, age, n, hard_pm=hard_pm, stable_pm=stable_pm, seed=n)
        assert got.sum() == n
        if kh + ks == n:                               # no uniform remainder to blur the groups
            assert got[:n].sum() == kh and got[n:2 * n].sum() == ks, (n, kh, ks)
        else:
            assert got[:n].sum() >= kh and got[n:2 * n].sum() >= ks


def test_topk_age_brute_force(orc):
    rng = np.random.default_rng(2)
    for trial in range(50):
        cnt = int(rng.integers(1, 60))
        age = rng.integers(0, 5, cnt).astype(np.uint32)     # many ties
        n = int(rng.integers(0, cnt + 1))
        got = orc.choose_items(np.zeros(cnt, np.uint64), age, n, hard_pm=0, stable_pm=1000, seed=trial)
        order = sorted(range(cnt), key=lambda i: (-int(age[i]), i))
        want = np.zeros(cnt, bool)
        want[order[:n]] = True
        np.testing.assert_array_equal(got, want)


def test_single_weighted_draw_frequency(orc):
    w = np.array([1, 2, 3, 4, 10, 0, 5], np.uint64) * 7
    age = np.zeros(7, np.uint32)
    N = 20000
    hits = np.zeros(7)
    for s in range(N):
        hits += orc.choose_items(w, age, 1, hard_pm=1000, stable_pm=0, seed=s)
    p = w.astype(float) / w.sum()
    chi2 = ((hits - N * p) ** 2 / np.maximum(N * p, 1e-9))[p > 0].sum()
    assert hits[5] == 0
    assert chi2 < 22.5                     # chi-square, 5 dof, p ~ 4e-4


def test_weighted_inclusion_matches_successive_draws(orc):
    w = np.array([1, 3, 6, 10], np.uint64)
    p = w.astype(float) / w.sum()
    want = _seq_inclusion(p, 2)
    N = 30000
    hits = np.zeros(4)
    for s in range(N):
        hits += orc.choose_items(w, np.zeros(4, np.uint32), 2, hard_pm=1000, stable_pm=0, seed=s, it=7)
    np.testing.assert_allclose(hits / N, want, atol=0.012)


def test_zero_weights_fall_back_to_uniform(orc):
    N = 12000
    hits = np.zeros(6)
    for s in range(N):
        hits += orc.choose_items(np.zeros(6, np.uint64), np.zeros(6, np.uint32), 2, hard_pm=1000, stable_pm=0,
                                 seed=s)
    np.testing.assert_allclose(hits / N, 2 / 6, atol=0.02)


def test_uniform_remainder(orc):
    N = 12000
    hits = np.zeros(8)
    w = np.arange(8, dtype=np.uint64)
    for s in range(N):
        hits += orc.choose_items(w, np.zeros(8, np.uint32), 3, hard_pm=0, stable_pm=0, seed=s, tile=5)
    np.testing.assert_allclose(hits / N, 3 / 8, atol=0.02)


def test_three_way_split(orc):
    """Positive weight on exactly k_hard items: the draw takes them; the
    oldest k_stable of the rest follow; the rest are uniform."""
    cnt, n = 40, 20
    kh, ks = (400 * n + 500) // 1000, (300 * n + 500) // 1000
    rng = np.random.default_rng(4)
    for s in range(20):
        w = np.zeros(cnt, np.uint64)
        hard = rng.choice(cnt, kh, replace=False)
        w[hard] = rng.integers(1, 100, kh).astype(np.uint64)
        age = rng.permutation(cnt).astype(np.uint32)
        got = orc.choose_items(w, age, n, seed=s)
        assert got.sum() == n and got[hard].all()
        rest = [i for i in range(cnt) if i not in set(hard)]
        oldest = sorted(rest, key=lambda i: -int(age[i]))[:ks]
        assert got[oldest].all()


def test_select_structure(orc):
    for (W, H, n_sel, n_pix) in [(256, 256, 64, 256), (200, 130, 20, 25), (200, 130, 1000, 84),
                                 (40, 40, 1, 1), (37, 21, 3, 256), (64, 64, 0, 10)]:
        err = scenes.error_map(W, H, seed=W)
        age = scenes.age_map(W, H, seed=H)
        sel = orc.select(err, age, W, H, n_select=n_sel, n_pix=n_pix, seed=11, it=3)
        tx_n, ty_n = (W + 15) // 16, (H + 15) // 16
        T = tx_n * ty_n
        A = sel["n_active"]
        assert A == min(n_sel, T)
        act = sel["active_tiles"]
        assert np.all(np.diff(act) > 0)
        np.testing.assert_array_equal(sel["tile_rank"][act], np.arange(A))
        assert (sel["tile_rank"] >= 0).sum() == A
        off = sel["pix_off"]
        for j, t in enumerate(act):
            tx, ty = t % tx_n, t // tx_n
            valid = min(16, W - 16 * tx) * min(16, H - 16 * ty)
            assert off[j + 1] - off[j] == min(n_pix, valid)
            loc = sel["pix_idx"][off[j]:off[j + 1]].astype(int)
            assert np.all(np.diff(loc) > 0)
            assert np.all(16 * tx + loc % 16 < W) and np.all(16 * ty + loc // 16 < H)
        again = orc.select(err, age, W, H, n_select=n_sel, n_pix=n_pix, seed=11, it=3)
        for k in ("active_tiles", "pix_off", "pix_idx"):
            np.testing.assert_array_equal(sel[k], again[k])


def test_hard_pixels_follow_error(orc):
    """One hard draw per tile picks pixel p with probability E(p) / sum E, so
    the mean picked error of a tile is sum E^2 / sum E (size-biased mean)."""
    W = H = 64
    err = np.random.default_rng(2).exponential(0.1, (H, W)).astype(np.float16).view(np.uint16)
    age = np.zeros((H, W), np.uint16)
    e = err.view(np.float16).astype(float)
    tiles = e.reshape(4, 16, 4, 16).transpose(0, 2, 1, 3).reshape(16, 256)
    want = ((tiles ** 2).sum(1) / tiles.sum(1)).mean()
    got = []
    for s in range(300):
        sel = orc.select(err, age, W, H, n_select=16, n_pix=1, pix_hard_pm=1000, pix_stable_pm=0, seed=s)
        P = orc.pixel_coords(sel["active_tiles"], sel["pix_off"], sel["pix_idx"], W)
        got.append(e[P[:, 1], P[:, 0]].mean())
    assert abs(np.mean(got) - want) < 0.03 * want
    assert want > 1.5 * e.mean()


def test_tile_age_is_the_smallest_pixel_age(orc):
    """A tile's age is its smallest pixel age (the iterations since any of its
    pixels was sampled): a tile with one very old pixel among fresh ones is
    younger than a tile whose pixels are all moderately old."""
    W, H = 64, 16                                   # tiles 0..3 in one row
    age = np.full((H, W), 2, np.uint16)
    age[5, 3] = 900                                 # tile 0: one old pixel, the rest age 2
    age[:, 16:32] = 40                              # tile 1: every pixel age 40
    err = np.zeros((H, W), np.uint16)
    sel = orc.select(err, age, W, H, n_select=1, n_pix=4, tile_hard_pm=0, tile_stable_pm=1000)
    assert sel["active_tiles"].tolist() == [1]

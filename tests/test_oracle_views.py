"""Pins of the oracle's view sampling and schedule (Sec. 3.4 Eqs. 5-6; App. A
Eqs. 15-16): the exact error totals against numpy's own fp16 decoding, the
integer logarithm against math.log2, camera poses against the look-at
construction, the anchor as brute-force argmax, the stack's
without-replacement cycle, inclusion frequencies of the K - 1 draws against
exact enumeration of successive draws proportional to Eq. 6's weights, and
the schedule's end points, monotonicity and constant pixel budget.  The
host schedule of the library is checked against the oracle's."""
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


def _f16_maps(rng, V, H, W, specials=True):
    x = rng.exponential(0.05, size=(V, H, W)).astype(np.float16)
    if specials:
        flat = x.reshape(-1)
        idx = rng.choice(flat.size, size=min(40, flat.size), replace=False)
        vals = np.array([-0.5, np.nan, np.inf, -np.inf, 6.0e-8, 65504.0, 0.0, -0.0], np.float16)
        flat[idx] = vals[np.arange(idx.size) % vals.size]
    return x


def test_error_sums_match_numpy_decoding(orc):
    rng = np.random.default_rng(0)
    for V, H, W in ((1, 1, 1), (3, 7, 5), (4, 33, 17)):
        x = _f16_maps(rng, V, H, W)
        got = orc.view_error_sums(x.view(np.uint16))
        v = x.astype(np.float64)
        v[~np.isfinite(v) | (v < 0)] = 0.0
        want = (v * 2.0 ** 24).astype(np.int64).reshape(V, -1).sum(1)   # every fp16 * 2^24 is an integer
        np.testing.assert_array_equal(got.astype(np.int64), want)


def test_error_sums_constant_map(orc):
    x = np.full((2, 9, 11), 0.375, np.float16)
    got = orc.view_error_sums(x.view(np.uint16))
    assert list(got) == [int(0.375 * 2 ** 24) * 99] * 2


@pytest.mark.parametrize("x", [1, 2, 3, 5, 1000, 2 ** 32, 2 ** 40 + 12345, 2 ** 64 - 1])
def test_log2_q32_against_math(orc, x):
    got = orc.log2_q32(x) / 2.0 ** 32
    want = math.log2(x)
    assert want - 4e-9 <= got <= want + 1e-12    # truncated digits: never above, a few 2^-32 below
    if x & (x - 1) == 0:
        assert orc.log2_q32(x) == (x.bit_length() - 1) << 32


def test_view_pose_matches_look_at(orc):
    for pos, tgt in (((0.0, 0.0, -4.0), (0.0, 0.0, 0.0)), ((3.0, -1.0, 2.0), (0.5, 0.2, -0.3)),
                     ((-2.0, 5.0, 1.0), (1.0, 1.0, 1.0))):
        cam = scenes.look_at(pos, tgt)
        c, d = orc.view_pose(np.asarray(cam["viewmat"]).reshape(16))
        f = np.subtract(tgt, pos)
        np.testing.assert_allclose(c, pos, atol=1e-5)
        np.testing.assert_allclose(d, f / np.linalg.norm(f), atol=1e-6)
        assert abs(np.linalg.norm(d) - 1.0) < 1e-15


def _cams(V, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(V):
        pos = rng.normal(size=3) * 3.0
        out.append(np.asarray(scenes.look_at(pos, rng.normal(size=3) * 0.2)["viewmat"], np.float32).reshape(16))
    return np.stack(out)


def test_anchor_is_the_argmax_of_mean_error(orc):
    rng = np.random.default_rng(1)
    vm = _cams(12)
    for trial in range(20):
        sums = rng.integers(0, 50, 12).astype(np.uint64)   # ties likely
        views, _ = orc.sample_views(sums, vm, 4, 1.0, 2.0, seed=trial)
        best = max(range(12), key=lambda v: (int(sums[v]), -v))
        assert views[0] == best
        assert len(set(views.tolist())) == 4


def test_stack_cycle_without_replacement(orc):
    V, K = 10, 3
    vm = _cams(V, 2)
    sums = np.arange(V, dtype=np.uint64) * 7
    stack = None
    seen = []
    for it in range(3):
        views, stack = orc.sample_views(sums, vm, K, 0.5, 1.0, seed=5, it=it, stack=stack)
        seen += views.tolist()
        assert stack.sum() == V - K * (it + 1)
    assert len(set(seen)) == 9                        # no view twice within a cycle
    # one view left (< K): the stack is refilled before the fourth draw
    views, stack = orc.sample_views(sums, vm, K, 0.5, 1.0, seed=5, it=3, stack=stack)
    assert views[0] == V - 1 and stack.sum() == V - K
    # K = V: every view, every time
    views, st = orc.sample_views(sums, vm, V, 0.5, 1.0, seed=1)
    assert sorted(views.tolist()) == list(range(V)) and st.sum() == 0


def _weights(vm, anchor, lam_d, lam_t):
    ca, da = (np.asarray(x) for x in scenes_pose(vm[anchor]))
    w = []
    for u in range(len(vm)):
        c, d = scenes_pose(vm[u])
        w.append(math.exp(-lam_d * np.linalg.norm(c - ca) - lam_t * (1.0 - float(np.dot(d, da)))))
    return np.array(w)


def scenes_pose(viewmat):
    M = np.asarray(viewmat, np.float64).reshape(4, 4)
    f = M[2, :3]
    return -M[:3, :3].T @ M[:3, 3], f / np.linalg.norm(f)


@pytest.mark.parametrize("lam_d,lam_t", [(0.6, 0.0), (0.0, 3.0), (0.4, 1.5), (0.0, 0.0)])
def test_draw_inclusion_matches_successive_draws(orc, lam_d, lam_t):
    vm = _cams(5, 3)
    sums = np.array([100, 1, 2, 3, 4], np.uint64)          # anchor: view 0
    w = _weights(vm, 0, lam_d, lam_t)[1:]
    want = _seq_inclusion(w / w.sum(), 2)
    N = 20000
    hits = np.zeros(4)
    for s in range(N):
        views, _ = orc.sample_views(sums, vm, 3, lam_d, lam_t, seed=s, it=11)
        assert views[0] == 0
        hits[views[1:] - 1] += 1
    np.testing.assert_allclose(hits / N, want, atol=0.012)


def test_single_draw_frequency_follows_eq6(orc):
    vm = _cams(6, 4)
    sums = np.array([0, 0, 9, 0, 0, 0], np.uint64)          # anchor: view 2
    lam_d, lam_t = 0.5, 2.0
    w = np.delete(_weights(vm, 2, lam_d, lam_t), 2)
    p = w / w.sum()
    N = 20000
    hits = np.zeros(5)
    for s in range(N):
        views, _ = orc.sample_views(sums, vm, 2, lam_d, lam_t, seed=s)
        u = int(views[1])
        hits[u if u < 2 else u - 1] += 1
    chi2 = ((hits - N * p) ** 2 / (N * p)).sum()
    assert chi2 < 20.5                                       # chi-square, 4 dof, p ~ 4e-4


def test_schedule_end_points_and_budget(orc):
    # start with the initial error: g = 0, every view at the lowest rate
    K, r = orc.sampling_schedule(0, 0.7, 0.7)
    assert K == 10 and r == pytest.approx(1.0 / 10)
    # from tau_until on (or with no error left) g = 1: K_min + 7 e^-3 rounds to 3
    for args in ((3500, 0.7, 0.7), (9000, 0.1, 0.7), (0, 0.0, 0.7)):
        K, r = orc.sampling_schedule(*args)
        assert K == 3 and r == pytest.approx(1.0 / 3)
    # phi(1/4) = sin(pi/4): g = 1 - sqrt(2)/2 at t = 0
    K, r = orc.sampling_schedule(0, 0.25, 1.0)
    g = 1.0 - math.sqrt(0.5)
    assert r == pytest.approx(0.1 + (1.0 / 3 - 0.1) * g, rel=1e-7)
    # the ratio is clipped: more error than at the start counts as the start
    assert orc.sampling_schedule(100, 5.0, 1.0) == orc.sampling_schedule(100, 1.0, 1.0)


def test_schedule_monotone(orc):
    prev = None
    for t in range(0, 4001, 50):
        K, r = orc.sampling_schedule(t, 0.6, 1.0)
        if prev:
            assert K <= prev[0] and r >= prev[1] - 1e-15
        prev = (K, r)
    prev = None
    for e in np.linspace(0.0, 1.0, 41):
        K, r = orc.sampling_schedule(1000, float(e), 1.0)
        if prev:
            assert K >= prev[0] and r <= prev[1] + 1e-15
        prev = (K, r)


def test_library_schedule_matches_oracle(orc):
    from paper_2606_15924_gb300.config import ScheduleConfig
    from paper_2606_15924_gb300.views import pixels_per_tile, sampling_schedule
    rng = np.random.default_rng(9)
    for _ in range(300):
        t = int(rng.integers(0, 6000))
        e0 = float(rng.uniform(0.01, 1.0))
        e = float(rng.uniform(0.0, 1.5)) * e0
        lam = float(rng.uniform(0.1, 1.0))
        s = ScheduleConfig(lam=lam)
        K, r = sampling_schedule(t, e, e0, s)
        Ko, ro = orc.sampling_schedule(t, e, e0, K_max=s.K_max, K_min=s.K_min, alpha=s.alpha,
                                       tau_until=s.tau_until, lam=lam)
        assert K == Ko and r == pytest.approx(ro, rel=1e-12)
        assert 1 <= pixels_per_tile(r) <= 256
    assert pixels_per_tile(1.0 / 3) == 85 and pixels_per_tile(0.0) == 1 and pixels_per_tile(2.0) == 256


def test_library_camera_pose_matches_oracle(orc):
    from paper_2606_15924_gb300.views import camera_pose
    vm = _cams(8, 6)
    for m in vm:
        c, d = camera_pose(dict(viewmat=m.reshape(4, 4)))
        co, do = orc.view_pose(m)
        np.testing.assert_allclose(c, co, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(d, do, rtol=1e-12, atol=1e-12)

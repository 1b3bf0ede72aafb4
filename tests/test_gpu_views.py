"""GPU parity of geometry-aware view sampling (Sec. 3.4, Eqs. 5-6): the exact
per-view error totals and the K-view draw with its stack, bit for bit against
the oracle on the same seeded error maps, cameras and hash seeds."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2606_15924_gb300 import binding
    binding.device_check()
    return binding


def _maps(V, H, W, seed):
    rng = np.random.default_rng(seed)
    x = rng.exponential(0.05, size=(V, H, W)).astype(np.float16)
    flat = x.reshape(-1)
    idx = rng.choice(flat.size, size=min(64, flat.size), replace=False)
    vals = np.array([-0.5, np.nan, np.inf, -np.inf, 6.0e-8, 65504.0, 0.0, -0.0], np.float16)
    flat[idx] = vals[np.arange(idx.size) % vals.size]
    return x.view(np.uint16)


def _gpu_sums(B, maps):
    d = torch.from_numpy(maps.view(np.int16)).cuda()
    s = torch.full((maps.shape[0],), -1, dtype=torch.int64, device="cuda")
    B.view_error_sums(d, s)
    return s.cpu().numpy().view(np.uint64)


# (V, H, W): 16-byte path when H W is a multiple of 8, else one value per thread
SUM_CASES = [(1, 1, 1), (3, 7, 5), (5, 33, 17), (2, 8, 8), (4, 720, 1280), (1, 1080, 1920), (300, 9, 13)]


@pytest.mark.parametrize("V,H,W", SUM_CASES)
def test_error_sums_bit_exact(B, orc, V, H, W):
    maps = _maps(V, H, W, V * 7 + H)
    np.testing.assert_array_equal(_gpu_sums(B, maps), orc.view_error_sums(maps))


def test_error_sums_full_size(B, orc):
    """256 views of 1280 x 720, the measured configuration."""
    rng = np.random.default_rng(5)
    maps = rng.exponential(0.05, size=(256, 720, 1280)).astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(_gpu_sums(B, maps), orc.view_error_sums(maps))


def _cams(V, seed):
    rng = np.random.default_rng(seed)
    cams = [scenes.look_at(rng.normal(size=3) * 3.0, rng.normal(size=3) * 0.2, width=64, height=48)
            for _ in range(V)]
    vm = np.stack([np.asarray(c["viewmat"], np.float32).reshape(16) for c in cams])
    return cams, vm


# (V, K, lambda_d, lambda_theta, draws)
DRAW_CASES = [
    (1, 1, 1.0, 2.0, 3),
    (7, 3, 0.5, 2.0, 8),        # refills every other draw
    (64, 10, 0.7, 2.0, 12),
    (1024, 10, 0.4, 1.0, 4),    # one view per thread
    (1025, 10, 0.4, 1.0, 4),    # two per thread
    (3000, 8, 0.2, 3.0, 3),     # four per thread
    (8192, 16, 0.3, 2.0, 2),    # eight per thread, the maximum
    (50, 50, 1.0, 1.0, 2),      # K = V
    (40, 1, 1.0, 1.0, 5),       # anchor only
    (40, 6, 0.0, 0.0, 5),       # uniform draw
]


@pytest.mark.parametrize("V,K,lam_d,lam_t,draws", DRAW_CASES)
def test_sample_views_bit_exact(B, orc, V, K, lam_d, lam_t, draws):
    rng = np.random.default_rng(V + K)
    cams, vm = _cams(V, V)
    sums = rng.integers(0, 40, V).astype(np.uint64) * np.uint64(1 << 20)    # ties between views
    cams_d = B.camera_array(cams)
    sums_d = torch.from_numpy(sums.view(np.int64)).cuda()
    stack_d = torch.ones(V, dtype=torch.uint8, device="cuda")
    views_d = torch.full((K,), -1, dtype=torch.int32, device="cuda")
    stack = np.ones(V, np.uint8)
    for it in range(draws):
        B.sample_views(sums_d, cams_d, K, lam_d, lam_t, 17, it, stack_d, views_d)
        want, stack = orc.sample_views(sums, vm, K, lam_d, lam_t, seed=17, it=it, stack=stack)
        np.testing.assert_array_equal(views_d.cpu().numpy(), want)
        np.testing.assert_array_equal(stack_d.cpu().numpy(), stack)


def test_sums_then_draw(B, orc):
    """The two calls chained on the device, as ViewSampler runs them."""
    from paper_2606_15924_gb300.views import ViewSampler
    V = 48
    cams, vm = _cams(V, 3)
    maps = _maps(V, 48, 64, 3)
    vs = ViewSampler(cams, lambda_d=0.8, lambda_theta=2.0, seed=4)
    vs.error_sums(torch.from_numpy(maps.view(np.int16)).cuda())
    sums = orc.view_error_sums(maps)
    stack = None
    for it in range(6):
        got = vs.draw(5, it).cpu().numpy()
        want, stack = orc.sample_views(sums, vm, 5, 0.8, 2.0, seed=4, it=it, stack=stack)
        np.testing.assert_array_equal(got, want)
    np.testing.assert_allclose(vs.mean_errors(), sums.astype(np.float64) / 2 ** 24 / (48 * 64), rtol=1e-15)


def test_invalid_arguments(B):
    cams, _ = _cams(4, 1)
    cams_d = B.camera_array(cams)
    sums = torch.zeros(4, dtype=torch.int64, device="cuda")
    stack = torch.ones(4, dtype=torch.uint8, device="cuda")
    views = torch.zeros(8, dtype=torch.int32, device="cuda")
    for k, ld, lt in ((5, 1.0, 1.0), (0, 1.0, 1.0), (2, -1.0, 1.0), (2, 1.0, float("nan")), (2, float("inf"), 1.0)):
        with pytest.raises(B.TgsError) as e:
            B.sample_views(sums, cams_d, k, ld, lt, 0, 0, stack, views)
        assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.TgsError):
        B.view_error_sums(torch.zeros(1, 4096, 4096, dtype=torch.int16, device="cuda"), sums)   # > 2^23 pixels
    torch.cuda.synchronize()
    assert stack.cpu().numpy().tolist() == [1, 1, 1, 1]


def _pool_scene(V, W, H, n=6000):
    from gpu_util import gaussians_dev
    from paper_2606_15924_gb300.pipeline import Trainer
    from paper_2606_15924_gb300.quality import perturbed_init
    gt_np = scenes.gaussians(n, seed=0)
    gt = gaussians_dev(gt_np)
    cams = scenes.orbit(V, 4.0, W, H)
    targets = []
    for c in cams:
        d = Trainer(gt, c, torch.zeros(H, W, 3, device="cuda"), dense=True, train=False)
        d.forward()
        targets.append(d.scatter_image(d.rgb).contiguous())
    return gaussians_dev(perturbed_init(gt_np, 1.0)), cams, targets


def test_set_views_matches_a_fixed_trainer(B):
    """A pool trainer after set_views renders and scores its active views
    exactly as a trainer built for those views alone (same view ids, maps and
    pixels per tile)."""
    from paper_2606_15924_gb300.batched import MultiViewTrainer
    W, H = 128, 96
    g, cams, targets = _pool_scene(6, W, H)
    maps = [torch.from_numpy(scenes.error_map(W, H, seed=k).view(np.int16)).cuda() for k in range(6)]
    pool = MultiViewTrainer(g, cams, targets, [0.3] * 6, pixel_rate=0.34, max_active=3)
    for k, v in enumerate(pool.pool):
        v.err_map.copy_(maps[k])
    ids = [4, 1, 2]
    pool.set_views(ids, n_pix=20)
    fixed = MultiViewTrainer(g, [cams[i] for i in ids], [targets[i] for i in ids], [0.3] * 3,
                             pixel_rate=20.5 / 256, view_ids=ids)
    for k, v in enumerate(fixed.views):
        v.err_map.copy_(maps[ids[k]])
    for mv in (pool, fixed):
        mv.forward()
        mv.loss_and_maps()
    torch.cuda.synchronize()
    for a, b in zip(pool.views, fixed.views):
        assert a.n_pix == b.n_pix == 20
        P = int(b.pix_off[int(b.n_active.item())].item())
        assert P > 0
        assert torch.equal(a.pix_idx[:P], b.pix_idx[:P])
        assert torch.equal(a.rgb[:P], b.rgb[:P]) and torch.equal(a.T_final[:P], b.T_final[:P])
        assert float(a.loss.item()) == pytest.approx(float(b.loss.item()), rel=1e-6)
    with pytest.raises(ValueError):
        pool.set_views([0, 1, 2, 3])             # more than max_active
    with pytest.raises(ValueError):
        pool.set_views([1, 1])                   # repeated view
    with pytest.raises(ValueError):
        pool.set_views([0], n_pix=200)           # above the pool's allocation


def test_scheduled_trainer(B):
    """Alg. 1 steps 1-10 over a pool of 12 views: each iteration's K_t and
    pixels per tile follow the schedule of the measured mean errors, the
    views are a valid draw (distinct, from the stack, the anchor the stack
    view of largest error total, refills only when fewer than K_t remain),
    and training lowers the mean view error."""
    from paper_2606_15924_gb300.config import Config, ScheduleConfig
    from paper_2606_15924_gb300.views import ScheduledTrainer, pixels_per_tile, sampling_schedule
    W, H, V = 128, 96, 12
    g, cams, targets = _pool_scene(V, W, H)
    cfg = Config()
    cfg.schedule = ScheduleConfig(tau_until=30, K_max=5, K_min=2, alpha=3.0, lam=1.0)
    st = ScheduledTrainer(g, cams, targets, tile_fraction=0.3, cfg=cfg, seed=3)
    on = set(range(V))
    seen = set()
    for _ in range(40):
        rec = st.step()
        sums = st.sampler.sums.cpu().numpy()
        K, r = sampling_schedule(rec["t"], rec["E_t"], st.E_init, cfg.schedule)
        assert rec["K"] == K and rec["n_pix"] == pixels_per_tile(r)
        views = rec["views"]
        assert len(views) == K and len(set(views)) == K
        if len(on) < K:
            on = set(range(V))
        assert set(views) <= on
        assert views[0] == max(on, key=lambda v: (int(sums[v]), -v))
        on -= set(views)
        seen |= set(views)
    torch.cuda.synchronize()
    ks = [h["K"] for h in st.history]
    assert ks[0] == 5 and ks[-1] == 2             # g = 0 at the start; from tau_until on K_min + 3 e^-3 -> 2
    assert seen == set(range(V))
    assert st.history[-1]["E_t"] < st.E_init

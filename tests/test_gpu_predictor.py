"""Tile-error predictor on the GPU: the tile memory, feature and refresh
kernels against the oracle, and what the online-trained network gains over
the stale error maps of the plain method (scored by dense evaluations)."""
import math

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


def test_observe_features_refresh_parity(B, orc):
    rng = np.random.default_rng(3)
    W, H = 200, 130
    cam = scenes.look_at((0.0, 0.0, -4.0), width=W, height=H)
    T = ((W + 15) // 16) * ((H + 15) // 16)
    A_max, A = 40, 33
    active = np.sort(rng.choice(T, A, replace=False)).astype(np.int32)
    counts = rng.integers(1, 90, A)
    pix_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    P = int(pix_off[-1])
    Tf = rng.uniform(0, 1, P).astype(np.float32)
    err = rng.exponential(0.2, P).astype(np.float32)
    ranges = np.zeros((A_max, 2), np.int32)
    ranges[:A, 0] = np.arange(A) * 1000
    ranges[:A, 1] = ranges[:A, 0] + rng.integers(0, 900, A)
    d = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a)).cuda() if dt is None else \
        torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()
    at = torch.zeros(A_max, dtype=torch.int32, device="cuda")
    at[:A] = d(active)
    po = torch.zeros(A_max + 1, dtype=torch.int32, device="cuda")
    po[:A + 1] = d(pix_off)
    mem = torch.zeros(T, 4, device="cuda")
    mem_it = torch.zeros(T, dtype=torch.int64, device="cuda")
    target = torch.full((A_max,), -1.0, device="cuda")
    # features of the active rows before the observation, then the observation
    x_before = torch.empty(A_max, 16, device="cuda")
    n_act = torch.tensor([A], dtype=torch.int32, device="cuda")
    B.tile_features(mem, mem_it, cam, x_before, rows=at, n_rows=n_act, n_rows_max=A_max, view_cos=0.3, it=5)
    B.tile_observe(at, n_act, A_max, po, d(ranges), d(Tf), d(err), mem, mem_it, target, it=12)
    mem_o = np.zeros((T, 4))
    mem_it_o = np.zeros(T, dtype=np.int64)
    x_before_o = orc.tile_features(mem_o, mem_it_o, cam, rows=active, view_cos=0.3, iter_=5)
    tgt_o = orc.tile_observe(A, active, pix_off, ranges[:A], Tf, err, 12, mem_o, mem_it_o)
    # a second observation of the same tiles, as residuals
    err2 = (err * rng.uniform(0.5, 1.0, P)).astype(np.float32)
    target2 = torch.empty(A_max, device="cuda")
    mem_c, mem_it_c = mem.clone(), mem_it.clone()
    B.tile_observe(at, n_act, A_max, po, d(ranges), d(Tf), d(err2), mem_c, mem_it_c, target2, it=13,
                   residual=True)
    mem_o2, mem_it_o2 = mem_o.copy(), mem_it_o.copy()
    tgt_o2 = orc.tile_observe(A, active, pix_off, ranges[:A], Tf, err2, 13, mem_o2, mem_it_o2, residual=True)
    np.testing.assert_allclose(target2.cpu().numpy()[:A], tgt_o2, rtol=1e-4, atol=2e-6)
    np.testing.assert_allclose(x_before.cpu().numpy()[:A], x_before_o, rtol=1e-6, atol=1e-6)
    assert torch.all(x_before[A:] == 0)
    np.testing.assert_allclose(target.cpu().numpy()[:A], tgt_o, rtol=1e-5, atol=1e-6)
    assert torch.all(target[A:] == 0)
    np.testing.assert_allclose(mem.cpu().numpy(), mem_o, rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(mem_it.cpu().numpy(), mem_it_o)
    # features of every tile after the observation
    x_all = torch.empty(T, 16, device="cuda")
    B.tile_features(mem, mem_it, cam, x_all, view_cos=-0.2, it=30)
    x_all_o = orc.tile_features(mem_o, mem_it_o, cam, view_cos=-0.2, iter_=30)
    np.testing.assert_allclose(x_all.cpu().numpy(), x_all_o, rtol=1e-5, atol=1e-5)
    # refresh of an error map from predictions (one fp16 ulp)
    bits = scenes.error_map(W, H, seed=9)
    bits[0:16, 0:16] = 0
    pred = rng.uniform(-0.3, 1.2, T).astype(np.float32)
    e = d(bits.view(np.int16))
    B.tile_refresh(d(pred), e, W, H)
    got = e.cpu().numpy().view(np.float16).astype(np.float64)
    want = orc.tile_refresh(pred.astype(np.float64), bits, W, H).view(np.float16).astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=1.5e-3, atol=1e-7)
    e = d(bits.view(np.int16))
    B.tile_refresh(d(pred - 0.5), e, W, H, base=x_all)            # residual predictions on the stale value
    got = e.cpu().numpy().view(np.float16).astype(np.float64)
    want = orc.tile_refresh((pred - 0.5).astype(np.float64), bits, W, H,
                            base=x_all.cpu().numpy().astype(np.float64)).view(np.float16).astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=1.5e-3, atol=1e-7)


def _view_dir(cam):
    return np.asarray(cam["viewmat"], dtype=np.float64).reshape(4, 4)[2, :3]


def test_online_predictor_beats_stale_error_maps(B):
    """48 views share one scene (a perturbed copy of a ground-truth cloud,
    targets rendered from the truth); each step trains one randomly drawn view
    on 10% of its tiles with the plain sampler while the network learns from
    the step's measured tile errors, so most tiles of most views are long
    unobserved when they are scored - the regime of a large view set.  A dense
    evaluation of every third view (the plain refresh) then scores the
    per-tile estimates.  The network's estimates must be clearly closer to the
    truth than the stale error maps the plain method would select from, pick
    tiles holding about as much of the error, and cost a fraction of the
    dense refresh."""
    from paper_2606_15924_gb300.pipeline import Trainer
    from paper_2606_15924_gb300.predictor import TileErrorPredictor
    from paper_2606_15924_gb300.quality import perturbed_init
    W, H, V, n = 256, 192, 48, 60000
    gt = scenes.gaussians(n, seed=1)
    init = perturbed_init(gt, extent=1.0)
    cams = scenes.orbit(V, 4.0, W, H)
    gt_d = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in gt.items()}
    dummy = torch.zeros(H, W, 3, device="cuda")
    targets = [Trainer(gt_d, c, dummy, dense=True, train=False).render_image().contiguous() for c in cams]
    params = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in init.items()}
    trs = [Trainer(params, cams[v], targets[v], tile_fraction=0.1, view=v) for v in range(V)]
    shared = trs[0]
    for tr in trs[1:]:   # one optimiser state and one set of counters for the scene
        tr.grads, tr.m, tr.v, tr.touched = shared.grads, shared.m, shared.v, shared.touched
        tr.it_dev, tr.step_dev = shared.it_dev, shared.step_dev
    pred = TileErrorPredictor(min_batches=50)
    for tr in trs:
        pred.init_view(tr, it=0)
    rng = np.random.default_rng(0)
    prev = _view_dir(cams[0])
    steps = 400
    for it in range(1, steps + 1):
        v = int(rng.integers(V))
        tr = trs[v]
        cosv = float(np.dot(_view_dir(cams[v]), prev))
        tr.forward()
        tr.loss_and_maps()
        pred.observe_and_train(tr, it=it, view_cos=cosv)
        tr.backward()
        tr.update()
        B.advance_counters(tr.it_dev, tr.step_dev)
        prev = _view_dir(cams[v])
    torch.cuda.synchronize()
    assert pred.batches == steps and pred.recent_mse is not None
    mse_p, mse_s, mass_p, mass_s, mass_best = [], [], [], [], []
    for v, tr in list(enumerate(trs))[::3]:
        j = pred.assess(tr, it=steps + 1, view_cos=float(np.dot(_view_dir(cams[v]), prev)))
        mse_p.append(j["mse_pred"])
        mse_s.append(j["mse_stale"])
        truth = torch.expm1(j["truth"])
        k = truth.numel() // 4
        tot = float(truth.sum().item())
        for est, acc in ((j["pred"], mass_p), (j["stale"], mass_s), (j["truth"], mass_best)):
            # the estimates that pick the tiles
            acc.append(float(truth[torch.topk(est, k).indices].sum().item()) / tot)
    mp, ms = float(np.mean(mse_p)), float(np.mean(mse_s))
    print(f"\nlog-error MSE: predicted {mp:.4f}  stale {ms:.4f}; error mass in the top quarter of tiles: "
          f"predicted {np.mean(mass_p):.3f}  stale {np.mean(mass_s):.3f}  best {np.mean(mass_best):.3f}")
    assert mp < 0.6 * ms
    assert np.mean(mass_p) >= np.mean(mass_s) - 0.03
    # cost of a predicted refresh against the plain one (a dense render and
    # loss of the view with buffers already allocated), CUDA events
    tr = trs[0]
    d = Trainer(tr.params, tr.cam, tr.target, dense=True, train=False, view=0)
    x = pred.features(tr, steps + 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def predicted():
        B.tile_features(pred.memory(tr).mem, pred.memory(tr).it, tr.ccam, x, n_rows_max=tr.T, it=steps + 1)
        B.tile_refresh(pred.mlp.predict(x), tr.err_map, W, H, base=x)

    def plain():
        d.forward()
        d.loss_and_maps()
    t_pred, t_plain = timed(predicted), timed(plain)
    print(f"refresh of one {W}x{H} view: predicted {t_pred * 1e3:.1f} us, dense {t_plain * 1e3:.1f} us")
    assert t_pred < 0.5 * t_plain

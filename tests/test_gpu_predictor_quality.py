"""What the learned tile-error predictor gains, judged by held-out quality.

A view set large enough that error maps go stale: 48 views of one scene on an
orbit, every eighth held out (42 training views); each iteration trains one
drawn view on 10 % of its tiles, so a view is revisited about every 42
iterations and most of its tiles far less often.  Three arms train the same
start with the same view draws and the same sampler:

- ``none``: the error and age maps change only where a view's own steps
  sample (the method as the paper states it: the age map brings neglected
  pixels back, Sec. 3.3);
- ``plain``: a drawn view whose map was last refreshed REFRESH_AGE or more
  iterations ago is first refreshed by a dense evaluation of the view (every
  tile and pixel rendered and scored);
- ``predicted``: the same schedule, the refresh taken from the online-trained
  network's per-tile predictions once its recent error is low enough (the
  plain refresh before that), while the network trains on every step's tiles.

Held-out PSNR (foreground pixels, mean over the 6 held-out views) is taken
every EVAL iterations; the time axis is the host wall clock of the training
loop (eager launches, a wait for the device before each reading), with the
evaluations left out.  The test prints each arm's curve and the time each
takes to come within 0.1 dB of the plain arm's final PSNR, and checks what
holds by construction: the predicted arm reaches that quality, its refreshes
are mostly predicted and each costs less than a dense one."""
import time

import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu

W, H, V, HOLD, N = 256, 192, 48, 8, 60000
STEPS, EVAL, REFRESH_AGE = 1200, 150, 96


@pytest.fixture(scope="module")
def B():
    from paper_2606_15924_gb300 import binding
    binding.device_check()
    return binding


@pytest.fixture(scope="module")
def scene(B):
    from paper_2606_15924_gb300.quality import _gt_views, perturbed_init
    gt = scenes.gaussians(N, seed=1)
    init = perturbed_init(gt, extent=1.0)
    cams = scenes.orbit(V, 4.0, W, H)
    gt_d = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in gt.items()}
    targets, masks = _gt_views(gt_d, cams, noise=0.01, seed=3)
    del gt_d
    train = [v for v in range(V) if v % HOLD != HOLD - 1]
    held = [v for v in range(V) if v % HOLD == HOLD - 1]
    draws = np.random.default_rng(11).choice(train, STEPS + 1)
    return dict(init=init, cams=cams, targets=targets, masks=masks, train=train, held=held, draws=draws)


def _view_dir(cam):
    return np.asarray(cam["viewmat"], dtype=np.float64).reshape(4, 4)[2, :3]


def _run(B, sc, arm):
    from paper_2606_15924_gb300.pipeline import Trainer
    from paper_2606_15924_gb300.predictor import TileErrorPredictor
    from paper_2606_15924_gb300.quality import HeldOutEvaluator
    params = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in sc["init"].items()}
    cams, targets = sc["cams"], sc["targets"]
    trs = {}
    for v in sc["train"]:
        trs[v] = Trainer(params, cams[v], targets[v], tile_fraction=0.1, view=v,
                         share=next(iter(trs.values())) if trs else None)
    pred = TileErrorPredictor(min_batches=50, score_every=10) if arm == "predicted" else None
    for tr in trs.values():
        if pred is not None:
            pred.init_view(tr, it=0, want_loss=False)
        else:
            tr.init_error_map(want_loss=False)
    ev = HeldOutEvaluator(params, [cams[v] for v in sc["held"]], [targets[v] for v in sc["held"]],
                          [sc["masks"][v] for v in sc["held"]])
    last = {v: 0 for v in trs}
    refresh_s, n_refresh = 0.0, 0
    torch.cuda.synchronize()
    curve = [(0, 0.0, ev.psnr())]
    wall = 0.0
    prev = _view_dir(cams[sc["draws"][0]])
    t0 = time.perf_counter()
    for it in range(1, STEPS + 1):
        v = int(sc["draws"][it])
        tr = trs[v]
        cosv = float(np.dot(_view_dir(cams[v]), prev))
        if arm != "none" and it - last[v] >= REFRESH_AGE:
            r0 = time.perf_counter()
            if pred is None:
                tr.init_error_map(want_loss=False)
            else:
                pred.refresh(tr, it, view_cos=cosv)
            torch.cuda.synchronize()
            refresh_s += time.perf_counter() - r0
            n_refresh += 1
            last[v] = it
        tr.forward()
        tr.loss_and_maps()
        if pred is not None:
            pred.observe_and_train(tr, it=it, view_cos=cosv)
        if tr.fused:
            tr.render_backward()
            tr.backward_update()
        else:
            tr.backward()
            tr.update()
        B.advance_counters(tr.it_dev, tr.step_dev)
        prev = _view_dir(cams[v])
        if it % EVAL == 0:
            torch.cuda.synchronize()
            wall += time.perf_counter() - t0
            curve.append((it, wall * 1e3, ev.psnr()))
            t0 = time.perf_counter()
    assert not any(tr.overflowed() for tr in trs.values())
    return dict(curve=curve, refresh_ms=1e3 * refresh_s / max(n_refresh, 1), n_refresh=n_refresh,
                refreshes=dict(pred.refreshes) if pred is not None else None)


def test_predicted_refresh_against_plain_and_none(B, scene):
    from paper_2606_15924_gb300.quality import time_to
    res = {arm: _run(B, scene, arm) for arm in ("none", "plain", "predicted")}
    goal = res["plain"]["curve"][-1][2] - 0.1
    print(f"\nheld-out PSNR (foreground, {len(scene['held'])} views) every {EVAL} iterations; goal {goal:.2f} dB")
    for arm, r in res.items():
        pts = " ".join(f"{p:.2f}" for _, _, p in r["curve"])
        t = time_to(r["curve"], goal)
        print(f"{arm:9s} {pts} | {r['curve'][-1][1]:.0f} ms wall, to goal "
              f"{'-' if t is None else f'{t:.0f} ms'}; refreshes {r['n_refresh']} at {r['refresh_ms']:.2f} ms"
              f"{'' if r['refreshes'] is None else ' ' + str(r['refreshes'])}")
    p, q = res["plain"], res["predicted"]
    assert p["curve"][-1][2] > p["curve"][0][2] + 1.0           # training works at all
    assert time_to(q["curve"], goal) is not None                 # the predicted arm reaches the plain quality
    assert q["refreshes"]["predicted"] >= 0.5 * q["n_refresh"]   # the network is trusted for most refreshes
    assert q["refresh_ms"] < p["refresh_ms"]                      # and a refresh costs less than a dense one

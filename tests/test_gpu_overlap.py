"""The overlapped capture of the one-view step (``Trainer.capture(overlap=
True)``): each replay makes the next iteration's tile and pixel selection on
a second stream beside its backward and update, into the other of two sets
of selection buffers.  That selection must be exactly the one the plain step
would make at the start of the next iteration (the same error and age maps,
the same iteration counter), and training must follow the plain step's
course."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu

W, H = 256, 192
SEL = ("active_tiles", "n_active", "tile_rank", "pix_off", "pix_idx")


@pytest.fixture(scope="module")
def B():
    from paper_2606_15924_gb300 import binding
    binding.device_check()
    return binding


def _trainer(dense=False, frac=0.3, rate=1 / 3, seed=5):
    from gpu_util import gaussians_dev
    from paper_2606_15924_gb300.pipeline import Trainer
    g = gaussians_dev(scenes.gaussians(20000, seed=seed))
    cam = scenes.look_at((0.0, 0.0, -4.0), width=W, height=H)
    tgt = torch.from_numpy(scenes.smooth_image(W, H, seed=8)).cuda()
    tr = Trainer(g, cam, tgt, tile_fraction=frac, pixel_rate=rate, dense=dense)
    tr.init_error_map()
    return tr, g


def _eager_selection(tr):
    """The selection the plain step would make now, into scratch buffers."""
    cur = tr._selection()
    scratch = {k: torch.empty_like(v) for k, v in cur.items()}
    tr._use_selection(scratch)
    tr._select()
    tr._use_selection(cur)
    torch.cuda.synchronize()
    return scratch


@pytest.mark.parametrize("dense,frac,rate", [(False, 0.3, 1 / 3), (False, 1.0, 0.1), (True, 1.0, 1.0)])
def test_prefetched_selection_is_the_plain_one(B, dense, frac, rate):
    tr, _ = _trainer(dense, frac, rate)
    tr.capture(overlap=True)
    first = {k: v.clone() for k, v in tr.next_selection().items()}
    for it in range(6):
        if it == 0:      # the prologue's selection is the plain one too
            want = _eager_selection(tr)
            for k in SEL:
                assert torch.equal(first[k], want[k]), k
        tr.replay()
        torch.cuda.synchronize()
        nxt = tr.next_selection()
        assert nxt["active_tiles"].data_ptr() != tr.active_tiles.data_ptr()
        want = _eager_selection(tr)
        n = int(want["n_active"].item())
        assert n == int(nxt["n_active"].item()) and n > 0
        for k in SEL:
            assert torch.equal(nxt[k], want[k]), (it, k)


def test_overlapped_training_follows_the_plain_step(B):
    losses = []
    for overlap in (False, True):
        tr, g = _trainer(seed=6)
        tr.capture(overlap=overlap)
        ls = []
        for _ in range(20):
            tr.replay()
            ls.append(tr.loss.clone())
        torch.cuda.synchronize()
        losses.append([float(x.item()) for x in ls])
    a, b = (np.array(x) for x in losses)
    # the same selections and the same arithmetic; only the float atomics of
    # the render backward may order differently
    np.testing.assert_allclose(a[:5], b[:5], rtol=1e-4)
    assert b[-1] < b[0] and abs(a[-1] - b[-1]) <= 0.02 * a[-1]


def test_step_that_copies_its_target_in(B):
    """capture(overlap=True, target_host=..., loss_host=...): each replayed
    step copies the target in from pinned host memory on its own stream (the
    loss waits for it) and its loss out to pinned host memory.  With the
    device target cleared first, training must follow the step whose target
    is already on the device, and every step's loss must reach the host."""
    runs = []
    for copy in (False, True):
        tr, _ = _trainer(seed=7)
        host = tr.target.detach().cpu().pin_memory()
        loss_host = torch.full((1,), -1.0, dtype=torch.float64).pin_memory()
        tr.capture(overlap=True, target_host=host if copy else None, loss_host=loss_host if copy else None)
        if copy:
            tr.target.zero_()
        ls = []
        for _ in range(12):
            tr.replay(with_copy=copy)
            ls.append(tr.loss.clone())
            if copy:
                torch.cuda.synchronize()
                assert float(loss_host[0]) == float(ls[-1].item())  # this step's loss, in host memory
        torch.cuda.synchronize()
        runs.append([float(x.item()) for x in ls])
        if copy:
            assert torch.equal(tr.target.cpu(), host)
    a, b = (np.array(x) for x in runs)
    np.testing.assert_allclose(a[:4], b[:4], rtol=1e-4)
    assert abs(a[-1] - b[-1]) <= 0.02 * a[-1]

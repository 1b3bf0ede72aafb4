"""The split forward (several 32-position runs of a tile's list walked at
once, composed in list order) against the oracle's per-pixel render
(Sec. 3.6, Eq. 1) and against the sequential walk of the same library.

Each case renders with checkpoints, once per walk (1 = the sequential walk,
2 and 4 = the split walk of that many runs at once, 3 = the sequential walk
with every warp on its own, which must give the same bits as 1, 5 = two
threads per pixel, each half of every run walked at once), at 1, 3, 5 and 8
pixels per 32-lane warp.  Images and final
transmittances match the oracle within 1e-4 at every sampled pixel whose
decisions are not within rounding of a threshold; n_last matches exactly
there.  Against the sequential walk, the split walk's images agree to 1e-5,
n_last and each tile's last position exactly except where a pixel's
transmittance ends within rounding of the stopping value, and every
checkpoint the backward reads (slot c of a pixel that blends past position
32 (c + 1)) agrees to 1e-5.  An opaque scene, where most pixels stop early,
exercises the stop inside a run and the early exit of a tile's rounds."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu
MARGIN = 1e-4
W = H = 256


@pytest.fixture(scope="module")
def B():
    from paper_2606_15924_gb300 import binding
    binding.device_check()
    yield binding
    binding.set_forward_split(0)


def _scene(opaque):
    g = scenes.gaussians(4000, seed=21)
    g["log_scales"] += 0.8 if opaque else 1.0
    if opaque:
        g["opacity_logits"][:] = 3.0                      # o ~ 0.95: pixels saturate early
    cam = scenes.look_at((0.0, 0.0, -4.0), width=W, height=H)
    return g, cam


def _render(B, pd, binned, sel, n_pix, cam, slots):
    from gpu_util import dev
    P = sel["n_sel"] * n_pix
    out = dict(rgb=torch.zeros(P, 3, device="cuda"), T=torch.zeros(P, device="cuda"),
               n_last=torch.zeros(P, dtype=torch.int32, device="cuda"))
    data = torch.full((B.checkpoint_bytes(sel["n_sel"], n_pix, slots) // 4,), float("nan"), device="cuda")
    tl = torch.full((sel["n_sel"],), -1, dtype=torch.int32, device="cuda")
    ck = B.checkpoints(data, slots, sel["n_sel"] * n_pix, out["rgb"], tl)
    B.render_sampled(pd, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"], sel["n_sel"],
                     sel["pix_off"], sel["pix_idx"], n_pix, cam, (0.0, 0.0, 0.0), out["rgb"], out["T"],
                     out["n_last"], ckpt=ck)
    torch.cuda.synchronize()
    out["ck"] = data.view(slots, -1, 4).cpu().numpy()
    out["tile_last"] = tl.cpu().numpy()
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


@pytest.mark.parametrize("opaque", [False, True])
def test_split_forward_against_oracle_and_sequential(B, orc, opaque):
    from gpu_util import bin_dev, empty_projected, gaussians_dev, select_dev, select_host
    g, cam = _scene(opaque)
    n = g["means"].shape[0]
    err, age = scenes.error_map(W, H, seed=3), scenes.age_map(W, H, seed=4)
    g64 = {k: v.astype(np.float64) for k, v in g.items()}
    slots = 64
    stopped_seen = 0
    for n_select, n_pix in ((64, 25), (96, 85), (64, 150), (48, 256)):
        sel = select_dev(B, err, age, W, H, n_select, n_pix, seed=5)
        sh = select_host(sel)
        pd = empty_projected(n)
        B.project_gaussians(gaussians_dev(g), cam, sel["tile_rank"], pd)
        binned = bin_dev(B, pd, n, cam, sel["tile_rank"], sel["n_sel"], capacity=400000)
        P = int(sh["pix_off"][-1])
        A = sh["n_active"]
        outs = {}
        for groups in (1, 2, 3, 4, 5):
            B.set_forward_split(groups)
            outs[groups] = _render(B, pd, binned, sel, n_pix, cam, slots)
        B.set_forward_split(0)
        prw = orc.project(g64, cam, tile_rank=sh["tile_rank"])
        pix = orc.pixel_coords(sh["active_tiles"], sh["pix_off"], sh["pix_idx"], W)
        want = orc.render_pixels(prw, W, H, pix)
        sure = want["margin"] > MARGIN
        assert sure.mean() > 0.95
        seq = outs[1]
        stopped = seq["T"][:P] < 2e-4
        stopped_seen += int(stopped.sum())
        if not opaque:      # the longest walk spans several rounds
            assert seq["n_last"][:P].max() > 5 * 32
        # the warp-independent walk (3) takes the same per-pixel operations in the same order
        for k in ("rgb", "T", "n_last", "tile_last"):
            np.testing.assert_array_equal(outs[3][k], seq[k])
        np.testing.assert_array_equal(outs[3]["ck"][:, :P][np.isfinite(seq["ck"][:, :P])],
                                      seq["ck"][:, :P][np.isfinite(seq["ck"][:, :P])])
        for groups, o in outs.items():
            np.testing.assert_array_equal(o["n_last"][:P][sure], want["n_last"][sure])
            assert np.abs(o["rgb"][:P][sure] - want["rgb"][sure]).max() <= 1e-4, groups
            assert np.abs(o["T"][:P][sure] - want["T"][sure]).max() <= 1e-4, groups
            # against the sequential walk
            same = o["n_last"][:P] == seq["n_last"][:P]
            assert same.mean() > 0.998, groups
            assert np.abs(o["rgb"][:P] - seq["rgb"][:P])[same].max() <= 1e-5, groups
            assert np.abs(o["T"][:P] - seq["T"][:P])[same].max() <= 1e-5, groups
            assert (o["tile_last"][:A] == seq["tile_last"][:A]).mean() > 0.98, groups
            assert (o["tile_last"][:A] >= 0).all()
            # every checkpoint the backward reads
            nl = seq["n_last"][:P]
            for c in range(slots):
                rd = same & (nl > 32 * (c + 1))
                if not rd.any():
                    break
                assert np.abs(o["ck"][c, :P][rd] - seq["ck"][c, :P][rd]).max() <= 1e-5, (groups, c)
    if opaque:
        assert stopped_seen > 1000       # the stop inside a run is exercised


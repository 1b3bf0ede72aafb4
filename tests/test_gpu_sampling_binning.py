"""GPU parity of the integer steps: tile selection + pixel sampling and tile
binning are compared bit for bit with the oracle on the same seeded inputs."""
import numpy as np
import pytest

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2606_15924_gb300 import binding
    binding.device_check()
    return binding


SELECT_CASES = [
    # (W, H, n_select, n_pix, sampling)
    (256, 256, 64, 256, (400, 300, 400, 300)),     # tiny config: 25 % of tiles, every pixel
    (256, 256, 256, 256, (400, 300, 400, 300)),    # full mask
    (200, 130, 20, 25, (400, 300, 400, 300)),      # ragged tiles, rate 0.1
    (200, 130, 1000, 84, (400, 300, 400, 300)),    # n_select > tiles, rate 0.33
    (1280, 720, 360, 84, (400, 300, 400, 300)),    # 1280x720, 10 % of tiles
    (1280, 720, 1440, 25, (1000, 0, 1000, 0)),     # hard draws only
    (1280, 720, 720, 84, (0, 1000, 0, 1000)),      # oldest only
    (1280, 720, 720, 84, (0, 0, 0, 0)),            # uniform only
    (37, 21, 3, 1, (400, 300, 400, 300)),          # one pixel per tile, partial tiles
    (64, 64, 0, 10, (400, 300, 400, 300)),         # nothing selected
    (4096, 1040, 1664, 25, (400, 300, 400, 300)),  # 16 640 tiles: past the one-block selection (pairwise ranks)
]


@pytest.mark.parametrize("W,H,n_sel,n_pix,sampling", SELECT_CASES)
def test_select_bit_exact(B, orc, W, H, n_sel, n_pix, sampling):
    from gpu_util import select_dev, select_host
    err = scenes.error_map(W, H, seed=W + H)
    err[::7, ::5] = 0                                   # zero weights
    err[3, :4] = 0x8001                                # negative zero-ish / negative values count as 0
    age = scenes.age_map(W, H, seed=H, max_age=30)    # many age ties
    for it in (0, 5):
        got = select_host(select_dev(B, err, age, W, H, n_sel, n_pix, seed=123, it=it, view=2, sampling=sampling))
        want = orc.select(err, age, W, H, n_select=n_sel, n_pix=n_pix, tile_hard_pm=sampling[0],
                          tile_stable_pm=sampling[1], pix_hard_pm=sampling[2], pix_stable_pm=sampling[3], seed=123,
                          it=it, view=2)
        assert got["n_active"] == want["n_active"]
        np.testing.assert_array_equal(got["active_tiles"], want["active_tiles"])
        np.testing.assert_array_equal(got["tile_rank"], want["tile_rank"])
        np.testing.assert_array_equal(got["pix_off"], want["pix_off"])
        np.testing.assert_array_equal(got["pix_idx"], want["pix_idx"])


BIN_CASES = [
    # (n, W, H, mask fraction)
    (2000, 256, 256, None),
    (2000, 256, 256, 0.25),
    (30000, 1280, 720, 0.2),
    (5000, 200, 130, 0.5),        # ragged image
    (3000, 1600, 1060, None),     # > 256 tiles: two tile digits
]


@pytest.mark.parametrize("presort", [False, True])
@pytest.mark.parametrize("n,W,H,frac", BIN_CASES)
def test_bin_tiles_bit_exact(B, orc, n, W, H, frac, presort):
    from gpu_util import bin_dev, dev, projected_dev, tile_count
    pr = scenes.projected(n, W, H, seed=n + W)
    T = tile_count(W, H)
    rank = None
    n_active_max = T
    if frac is not None:
        rng = np.random.default_rng(5)
        act = rng.uniform(size=T) < frac
        rank = np.where(act, np.cumsum(act) - 1, -1).astype(np.int32)
        n_active_max = int(act.sum())
    want = orc.bin_tiles(pr["xy"], pr["radius"], pr["depth"], W, H, rank)
    keys_w, vals_w, counts_w = want
    cam = dict(viewmat=np.eye(4), fx=100.0, fy=100.0, cx=W / 2, cy=H / 2, width=W, height=H, znear=0.2)
    cap = max(len(vals_w) + 100, 2049 * T) if presort else len(vals_w) + 100
    out = bin_dev(B, projected_dev(pr), n, cam, None if rank is None else dev(rank), n_active_max, capacity=cap)
    I = int(out["n_isect"].item())
    assert I == len(vals_w)
    np.testing.assert_array_equal(out["vals"][:I].cpu().numpy(), vals_w)
    np.testing.assert_array_equal(out["keys"][:I].cpu().numpy().view(np.uint64), keys_w)
    # ranges per rank follow from the per-tile counts
    ranges = out["ranges"].cpu().numpy()
    tiles = np.arange(T) if rank is None else np.nonzero(rank >= 0)[0]
    starts = np.concatenate([[0], np.cumsum(counts_w[tiles])[:-1]])
    for r, t in enumerate(tiles):
        if counts_w[t] > 0:
            assert tuple(ranges[r]) == (starts[r], starts[r] + counts_w[t])
        else:
            assert ranges[r][1] - ranges[r][0] == 0


# Splats crowded into one tile, so that a tile's list is split into long
# runs: (total, crowded) -> every path of the per-segment sort (registers,
# warp shared memory, per-segment block sort, whole-range sort).
CLUSTER_CASES = [(5000, 5000), (50000, 50000), (200000, 30000), (200000, 200000)]


@pytest.mark.parametrize("presort", [False, True])
@pytest.mark.parametrize("n,n_crowd", CLUSTER_CASES)
def test_bin_tiles_crowded_tile_bit_exact(B, orc, n, n_crowd, presort):
    """presort: a capacity above 2048 pairs per tile makes bin_tiles sort the
    Gaussians by depth first and sort only segments of each tile's list."""
    from gpu_util import bin_dev, projected_dev
    W, H = 256, 256
    rng = np.random.default_rng(n + n_crowd)
    pr = scenes.projected(n, W, H, seed=n)
    xy = pr["xy"].copy()
    xy[:n_crowd] = rng.uniform(100.0, 110.0, size=(n_crowd, 2))
    pr["xy"] = xy.astype(np.float32)
    radius = pr["radius"].copy()
    radius[:n_crowd] = rng.integers(1, 6, n_crowd)
    pr["radius"] = radius.astype(np.int32)
    depth = pr["depth"].copy()
    depth[:n_crowd] = rng.uniform(1.0, 1.01, n_crowd)     # the crowd lies in front
    depth[:n_crowd:7] = depth[3]                         # with exact ties
    pr["depth"] = depth.astype(np.float32)
    keys_w, vals_w, counts_w = orc.bin_tiles(pr["xy"], pr["radius"], pr["depth"], W, H)
    assert counts_w.max() > 4096 or n_crowd < 20000
    cam = dict(viewmat=np.eye(4), fx=100.0, fy=100.0, cx=W / 2, cy=H / 2, width=W, height=H, znear=0.2)
    cap = max(len(vals_w) + 7, 2049 * 256) if presort else len(vals_w) + 7
    out = bin_dev(B, projected_dev(pr), n, cam, None, 256, capacity=cap)
    I = int(out["n_isect"].item())
    assert I == len(vals_w)
    np.testing.assert_array_equal(out["vals"][:I].cpu().numpy(), vals_w)
    np.testing.assert_array_equal(out["keys"][:I].cpu().numpy().view(np.uint64), keys_w)


# One tile's list grown through each size band of the per-tile sort (up to
# 256, 512, 1024, 2048 and 4096 keys in registers, and past 4096 in global
# memory), with exact depth ties.  presort: the same lists through the depth
# presort and the segment sort (whole list in shared memory up to 4096 keys,
# with segments sorted per lane, per warp and per block).
@pytest.mark.parametrize("presort", [False, True])
@pytest.mark.parametrize("n_crowd", [200, 300, 700, 1500, 3000, 3900, 4200])
def test_bin_tiles_sort_bands_bit_exact(B, orc, n_crowd, presort):
    from gpu_util import bin_dev, projected_dev
    W, H = 256, 256
    n = n_crowd + 500
    rng = np.random.default_rng(n_crowd)
    pr = scenes.projected(n, W, H, seed=n)
    xy = pr["xy"].copy()
    xy[:n_crowd] = rng.uniform(101.0, 107.0, size=(n_crowd, 2))   # inside tile (6, 6)
    pr["xy"] = xy.astype(np.float32)
    radius = pr["radius"].copy()
    radius[:n_crowd] = 1
    pr["radius"] = radius.astype(np.int32)
    depth = pr["depth"].copy()
    depth[:n_crowd] = rng.uniform(1.0, 1.01, n_crowd)
    depth[:n_crowd:5] = depth[2]                          # exact ties
    pr["depth"] = depth.astype(np.float32)
    keys_w, vals_w, counts_w = orc.bin_tiles(pr["xy"], pr["radius"], pr["depth"], W, H)
    assert counts_w.max() >= n_crowd
    cam = dict(viewmat=np.eye(4), fx=100.0, fy=100.0, cx=W / 2, cy=H / 2, width=W, height=H, znear=0.2)
    cap = max(len(vals_w) + 3, 2049 * 256) if presort else len(vals_w) + 3
    out = bin_dev(B, projected_dev(pr), n, cam, None, 256, capacity=cap)
    I = int(out["n_isect"].item())
    assert I == len(vals_w)
    np.testing.assert_array_equal(out["vals"][:I].cpu().numpy(), vals_w)
    np.testing.assert_array_equal(out["keys"][:I].cpu().numpy().view(np.uint64), keys_w)


def test_bin_tiles_edge_cases(B, orc):
    from gpu_util import bin_dev, projected_dev
    import torch
    W, H = 256, 256
    cam = dict(viewmat=np.eye(4), fx=100.0, fy=100.0, cx=128, cy=128, width=W, height=H, znear=0.2)
    # no Gaussians at all
    pr0 = scenes.projected(8, W, H)
    pr0 = {k: v[:0] for k, v in pr0.items()}
    out = bin_dev(B, projected_dev(pr0), 0, cam, None, 256, capacity=16)
    assert int(out["n_isect"].item()) == 0
    assert int(out["ranges"].abs().sum().item()) == 0
    # every Gaussian culled
    pr = scenes.projected(500, W, H, seed=4)
    pr["radius"][:] = 0
    out = bin_dev(B, projected_dev(pr), 500, cam, None, 256, capacity=16)
    assert int(out["n_isect"].item()) == 0
    # capacity too small: the true count is reported
    pr = scenes.projected(500, W, H, seed=4)
    want = orc.bin_tiles(pr["xy"], pr["radius"], pr["depth"], W, H)[1]
    out = bin_dev(B, projected_dev(pr), 500, cam, None, 256, capacity=10)
    assert int(out["n_isect"].item()) == len(want)
    # capacity 0 (the pair-count query): the count, and every range cleared
    ws = torch.empty(B.bin_tiles_workspace_size(500, 0, 256), dtype=torch.uint8, device="cuda")
    ranges = torch.full((256, 2), -1, dtype=torch.int32, device="cuda")
    n_isect = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    B.bin_tiles(projected_dev(pr), 500, cam, None, 256, ws, 0, None, None, ranges, n_isect)
    assert int(n_isect.item()) == len(want)
    assert int(ranges.abs().sum().item()) == 0
    torch.cuda.synchronize()


def test_invalid_arguments_are_rejected(B):
    import torch
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    e = torch.zeros(64, 64, dtype=torch.int16, device="cuda")
    with pytest.raises(B.TgsError) as ei:
        B.select_tiles(e, e, 64, 64, 4, 0, (400, 300, 400, 300), 0, 0, 0, ws, z, z, z, z,
                       torch.zeros(4, dtype=torch.uint8, device="cuda"))
    assert ei.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.TgsError):   # workspace too small
        B.select_tiles(e, e, 64, 64, 4, 10, (400, 300, 400, 300), 0, 0, 0, ws, z, z, z, z,
                       torch.zeros(40, dtype=torch.uint8, device="cuda"))

"""The allocation-free selection entry point, for callers that cannot allocate
device memory (a host that owns every device allocation through its own fixed
pool, or a latency-critical path where an allocation may block): it must
produce exactly what tgs_select_tiles produces with a caller workspace, on two
calls in a row (its built-in scratch keeps the previous call's contents), and
reject views larger than its fixed scratch.  Collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes

pytestmark = pytest.mark.gpu


def _buffers(W, H, n_select, n_pix):
    T = ((W + 15) // 16) * ((H + 15) // 16)
    n_sel = min(n_select, T)
    return dict(active_tiles=torch.full((max(n_sel, 1),), -3, dtype=torch.int32, device="cuda"),
                n_active=torch.zeros(1, dtype=torch.int32, device="cuda"),
                tile_rank=torch.zeros(T, dtype=torch.int32, device="cuda"),
                pix_off=torch.zeros(n_sel + 1, dtype=torch.int32, device="cuda"),
                pix_idx=torch.zeros(max(n_sel * n_pix, 1), dtype=torch.uint8, device="cuda"))


def _host(b):
    A = int(b["n_active"].item())
    off = b["pix_off"][:A + 1].cpu().numpy()
    return (A, b["active_tiles"][:A].cpu().numpy(), b["tile_rank"].cpu().numpy(), off,
            b["pix_idx"][:int(off[-1])].cpu().numpy())


CALLS = [  # two calls in a row with different sizes and seeds
    (1280, 720, 720, 84, 11, 3),
    (200, 130, 40, 25, 12, 4),
    (1280, 720, 360, 256, 13, 5),
]


def test_noalloc_matches_workspace_entry_point():
    from paper_2606_15924_gb300 import binding as B
    B.device_check()
    samp = (400, 300, 400, 300)
    for (W, H, n_select, n_pix, seed, it) in CALLS:
        err = torch.from_numpy(scenes.error_map(W, H, seed=seed).view(np.int16)).cuda()
        age = torch.from_numpy(scenes.age_map(W, H, seed=seed, max_age=40).view(np.int16)).cuda()
        ws = torch.empty(B.select_tiles_workspace_size(W, H), dtype=torch.uint8, device="cuda")
        want = _buffers(W, H, n_select, n_pix)
        B.select_tiles(err, age, W, H, n_select, n_pix, samp, seed, it, 0, ws, want["active_tiles"],
                       want["n_active"], want["tile_rank"], want["pix_off"], want["pix_idx"])
        got = _buffers(W, H, n_select, n_pix)
        B.select_tiles_noalloc(err, age, W, H, n_select, n_pix, samp, seed, it, 0, got["active_tiles"],
                               got["n_active"], got["tile_rank"], got["pix_off"], got["pix_idx"])
        torch.cuda.synchronize()
        for a, b in zip(_host(want), _host(got)):
            np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


def test_noalloc_rejects_views_beyond_its_scratch():
    from paper_2606_15924_gb300 import binding as B
    W, H = 4096, 1024 + 16            # 256 x 65 = 16640 tiles > 16384
    b = _buffers(W, H, 10, 10)
    err = torch.zeros(H, W, dtype=torch.int16, device="cuda")
    with pytest.raises(B.TgsError) as ei:
        B.select_tiles_noalloc(err, err, W, H, 10, 10, (400, 300, 400, 300), 0, 0, 0, b["active_tiles"],
                               b["n_active"], b["tile_rank"], b["pix_off"], b["pix_idx"])
    assert ei.value.status == B.ERR_CAPACITY

"""Helpers shared by the GPU parity tests: device buffers and calls through
the C ABI binding.  No arithmetic of the method lives here."""
import numpy as np
import torch


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gaussians_dev(g):
    n = g["means"].shape[0]
    return dict(means=dev(g["means"].astype(np.float32)), log_scales=dev(g["log_scales"].astype(np.float32)),
                quats=dev(g["quats"].astype(np.float32)),
                opacity_logits=dev(g["opacity_logits"].astype(np.float32)),
                sh=dev(np.asarray(g["sh"], np.float32).reshape(n, 16, 3)))


def empty_projected(n):
    return dict(xy=torch.zeros(n, 2, device="cuda"), conic_opac=torch.zeros(n, 4, device="cuda"),
                rgb=torch.zeros(n, 3, device="cuda"), depth=torch.zeros(n, device="cuda"),
                radius=torch.zeros(n, dtype=torch.int32, device="cuda"))


def projected_dev(p):
    """Screen-space splats from a numpy dict (xy, conic, opac, rgb, depth, radius)."""
    co = np.concatenate([p["conic"], p["opac"][:, None]], 1).astype(np.float32)
    return dict(xy=dev(p["xy"].astype(np.float32)), conic_opac=dev(co), rgb=dev(p["rgb"].astype(np.float32)),
                depth=dev(p["depth"].astype(np.float32)), radius=dev(p["radius"].astype(np.int32)))


def projected_host(pd):
    """Device projection -> numpy dict in the oracle's layout (float64)."""
    co = pd["conic_opac"].cpu().numpy().astype(np.float64)
    return dict(xy=pd["xy"].cpu().numpy().astype(np.float64), conic=co[:, :3], opac=co[:, 3],
                rgb=pd["rgb"].cpu().numpy().astype(np.float64), depth=pd["depth"].cpu().numpy().astype(np.float64),
                radius=pd["radius"].cpu().numpy())


def tile_count(W, H):
    return ((W + 15) // 16) * ((H + 15) // 16)


def select_dev(B, err, age, W, H, n_select, n_pix, seed=0, it=0, view=0, sampling=(400, 300, 400, 300)):
    T = tile_count(W, H)
    n_sel = min(n_select, T)
    ws = torch.empty(B.select_tiles_workspace_size(W, H), dtype=torch.uint8, device="cuda")
    out = dict(active_tiles=torch.full((max(n_sel, 1),), -7, dtype=torch.int32, device="cuda"),
               n_active=torch.zeros(1, dtype=torch.int32, device="cuda"),
               tile_rank=torch.zeros(T, dtype=torch.int32, device="cuda"),
               pix_off=torch.zeros(n_sel + 1, dtype=torch.int32, device="cuda"),
               pix_idx=torch.zeros(max(n_sel * n_pix, 1), dtype=torch.uint8, device="cuda"))
    B.select_tiles(dev(err), dev(age), W, H, n_select, n_pix, sampling, seed, it, view, ws, out["active_tiles"],
                   out["n_active"], out["tile_rank"], out["pix_off"], out["pix_idx"])
    out["n_sel"] = n_sel
    return out


def select_host(sel):
    A = int(sel["n_active"].item())
    off = sel["pix_off"][:A + 1].cpu().numpy()
    return dict(active_tiles=sel["active_tiles"][:A].cpu().numpy(), n_active=A,
                tile_rank=sel["tile_rank"].cpu().numpy(), pix_off=off,
                pix_idx=sel["pix_idx"][:int(off[-1]) if A > 0 else 0].cpu().numpy())


def bin_dev(B, proj_d, n, cam, tile_rank, n_active_max, capacity, want_keys=True):
    ws = torch.empty(B.bin_tiles_workspace_size(n, capacity, n_active_max), dtype=torch.uint8, device="cuda")
    vals = torch.zeros(max(capacity, 1), dtype=torch.int32, device="cuda")
    keys = torch.zeros(max(capacity, 1), dtype=torch.int64, device="cuda") if want_keys else None
    ranges = torch.zeros(max(n_active_max, 1), 2, dtype=torch.int32, device="cuda")
    n_isect = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.bin_tiles(proj_d, n, cam, tile_rank, n_active_max, ws, capacity, vals, keys, ranges, n_isect)
    return dict(vals=vals, keys=keys, ranges=ranges, n_isect=n_isect)


def render_dev(B, proj_d, binned, sel, n_pix, cam, bg=(0.0, 0.0, 0.0)):
    P = max(sel["n_sel"] * n_pix, 1)
    out = dict(rgb=torch.zeros(P, 3, device="cuda"), T=torch.zeros(P, device="cuda"),
               n_last=torch.zeros(P, dtype=torch.int32, device="cuda"))
    B.render_sampled(proj_d, binned["ranges"], binned["vals"], sel["active_tiles"], sel["n_active"], sel["n_sel"],
                     sel["pix_off"], sel["pix_idx"], n_pix, cam, bg, out["rgb"], out["T"], out["n_last"])
    return out

"""Argument checking of the C ABI, on the CPU.

Every entry point checks its arguments on the host before any CUDA call and
answers the invalid ones its header documents with TGS_ERR_INVALID_ARG (or
TGS_ERR_CAPACITY), so those calls are made here without a GPU.  Some cases
pass placeholder addresses that are never dereferenced; they run only where
no GPU is present (on a machine without one, a call that wrongly passed its
checks would fail with TGS_ERR_CUDA at its first CUDA call, not touch them).
Size queries and status strings are host functions."""
import ctypes as C
import math

import pytest
import torch

pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="host-side checks with placeholder addresses: CPU-only")

OK, INVALID, CAPACITY = 0, 1, 2
P16 = 0x1000          # placeholder, 16-byte aligned, never dereferenced


@pytest.fixture(scope="module")
def B():
    from paper_2606_15924_gb300 import build
    build.build()
    from paper_2606_15924_gb300 import binding
    return binding


def _defaults(fn):
    """Null pointers and zero scalars for every argument of fn."""
    out = []
    for t in fn.argtypes:
        if t in (C.c_double, C.c_float):
            out.append(0.0)
        elif t in (C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_size_t, C.c_int):
            out.append(0)
        else:
            out.append(None)
    return out


def _call(fn, **at):
    args = _defaults(fn)
    for k, v in at.items():
        args[int(k[1:])] = v
    return fn(*args)


def test_status_strings(B):
    names = [B._lib.tgs_status_string(k).decode() for k in range(6)]
    assert names[0] == "ok" and len(set(names)) == 6 and all(names)
    assert B._lib.tgs_status_string(99)
    assert B._lib.tgs_version().decode().startswith("turbogs-gb300")


def test_size_queries(B):
    L = B._lib
    assert L.tgs_select_tiles_workspace_size(0, 10) == 0
    assert L.tgs_select_tiles_workspace_size(1280, 720) > 0
    assert L.tgs_checkpoint_bytes(0, 85, 64) == 0 and L.tgs_checkpoint_bytes(720, 0, 64) == 0
    L.tgs_checkpoint_bytes.restype = C.c_size_t
    assert L.tgs_checkpoint_bytes(720, 85, 64) == 16 * 720 * 85 * 64
    assert L.tgs_bin_tiles_workspace_size(500000, 2000000, 720) > 0
    assert L.tgs_hybrid_step_workspace_size(500000) >= 4 * 500000
    assert L.tgs_mlp_backward_workspace_size(1000) > 0
    assert L.tgs_project_backward_multi_workspace_size(500000) >= 8 * 500000
    assert L.tgs_mlp_param_count() > 0


@pytest.mark.parametrize("name", [
    "tgs_select_tiles", "tgs_select_tiles_noalloc", "tgs_project_gaussians", "tgs_bin_tiles", "tgs_render_sampled",
    "tgs_loss_sparse_ncc", "tgs_backward_sampled", "tgs_render_backward_sampled", "tgs_error_stats_sampled",
    "tgs_project_backward", "tgs_project_backward_multi", "tgs_project_backward_update", "tgs_hybrid_step",
    "tgs_mlp_forward", "tgs_mlp_forward_tc", "tgs_mlp_backward", "tgs_mlp_train_tc", "tgs_mlp_adam", "tgs_mlp_tc_wait_drill",
    "tgs_tile_observe", "tgs_tile_features", "tgs_tile_refresh", "tgs_view_error_sums", "tgs_sample_views",
    "tgs_render_batched_resident", "tgs_advance_counters"])
def test_null_arguments_are_rejected(B, name):
    """Null pointers and zero sizes everywhere: the documented refusal."""
    fn = getattr(B._lib, name)
    assert fn.argtypes is not None, name
    assert _call(fn) == INVALID, name


def test_view_error_sums_checks(B):
    f = B._lib.tgs_view_error_sums   # (maps, V, stride, W, H, sums, stream)
    assert _call(f, a0=P16, a1=4, a2=4096 * 4096, a3=4096, a4=4096, a5=P16) == INVALID   # W H > 2^23
    assert _call(f, a0=P16, a1=0, a2=64, a3=8, a4=8, a5=P16) == INVALID                   # no views
    assert _call(f, a0=P16, a1=4, a2=63, a3=8, a4=8, a5=P16) == INVALID                   # stride < W H
    assert _call(f, a0=P16, a1=4, a2=64, a3=8, a4=8, a5=P16 + 4) == INVALID               # sums misaligned
    assert _call(f, a0=P16, a1=70000, a2=64, a3=8, a4=8, a5=P16) == INVALID               # grid rows


@pytest.mark.parametrize("V,K,ld,lt", [(10, 11, 1.0, 1.0), (10, 0, 1.0, 1.0), (8193, 4, 1.0, 1.0),
                                       (10, 3, -1.0, 1.0), (10, 3, 1.0, math.nan), (10, 3, math.inf, 1.0),
                                       (0, 1, 1.0, 1.0)])
def test_sample_views_checks(B, V, K, ld, lt):
    f = B._lib.tgs_sample_views      # (sums, cams, V, K, ld, lt, seed, iter, stack, views, stream)
    assert _call(f, a0=P16, a1=P16, a2=V, a3=K, a4=ld, a5=lt, a8=P16, a9=P16) == INVALID


def test_select_checks(B):
    cfg = B.Sampling(400, 300, 400, 300)
    f = B._lib.tgs_select_tiles_noalloc
    base = dict(a0=P16, a1=P16, a2=1280, a3=720, a4=100, a5=85, a6=C.byref(cfg), a11=P16, a12=P16, a13=P16,
                a14=P16, a15=P16)
    assert _call(f, **{**base, "a5": 0}) == INVALID                                # n_pix < 1
    assert _call(f, **{**base, "a5": 257}) == INVALID                              # n_pix > 256
    assert _call(f, **{**base, "a4": -1}) == INVALID                               # n_select < 0
    assert _call(f, **{**base, "a2": 4096, "a3": 1040}) == CAPACITY                # 16 640 tiles
    bad = B.Sampling(400, 700, 400, 1001)
    assert _call(f, **{**base, "a6": C.byref(bad)}) == INVALID                     # ratio above 1000


def test_render_checks(B):
    f = B._lib.tgs_render_sampled
    # n_pix_max outside 1..256 is refused before any pointer is looked at
    assert _call(f, a6=P16, a8=0) == INVALID
    assert _call(f, a6=P16, a8=257) == INVALID
    r = B._lib.tgs_render_batched_resident
    out = C.c_int32(0)
    assert r(0, 0, C.byref(out)) == INVALID
    assert r(85, 3, C.byref(out)) == INVALID


def test_hybrid_checks(B):
    f = B._lib.tgs_hybrid_step
    opt = B.Opt((C.c_float * 6)(*[1e-3] * 6), 0.9, 0.999, 1e-15, 1e-8, 1)
    assert _call(f, a10=C.byref(opt), a8=0) == INVALID                             # step < 1
    bad = B.Opt((C.c_float * 6)(*[1e-3] * 6), 1.0, 0.999, 1e-15, 1e-8, 1)
    assert _call(f, a10=C.byref(bad), a8=1) == INVALID                             # beta1 = 1
    bad = B.Opt((C.c_float * 6)(*[1e-3] * 6), 0.9, 0.999, 1e-15, 1e-8, 3)
    assert _call(f, a10=C.byref(bad), a8=1) == INVALID                             # mode 3


def test_forward_split_knob(B):
    """The forward's walk knob accepts 0 (automatic), 1 (sequential), 2 and 4
    (split), 3 (warp-independent) and 5 (two threads per pixel) only (no
    device work)."""
    f = B._lib.tgs_set_forward_split
    for bad in (-1, 6, 8):
        assert f(bad) == INVALID
    for ok in (1, 2, 3, 4, 5, 0):
        assert f(ok) == 0


def test_density_control_checks(B):
    """Density control refuses a bad configuration before any device work."""
    import torch
    f = B._lib.tgs_density_control
    g = B.Gaussians(None, None, None, None, None, 0, 3)
    pp = B.ParamPtrs(None, None, None, None, None)
    ws = (C.c_uint8 * 256)()
    n_out = C.c_int64(5)
    for bad in (B.density_params(0.5, 2e-4, -2.0, -5.3, topk_permille=1001),
                B.density_params(0.5, 2e-4, -2.0, -5.3, final_permille=-1),
                B.density_params(0.5, 2e-4, -2.0, -5.3, eps=-1.0)):
        assert f(C.byref(g), C.byref(pp), C.byref(pp), None, None, C.byref(bad), C.byref(pp), C.byref(pp),
                 C.byref(pp), 0, C.byref(n_out), None, ws, 256, None) == INVALID
    cfg = B.density_params(0.5, 2e-4, -2.0, -5.3)
    assert f(C.byref(g), C.byref(pp), C.byref(pp), None, None, None, C.byref(pp), C.byref(pp),
             C.byref(pp), 0, C.byref(n_out), None, ws, 256, None) == INVALID           # no configuration
    assert f(C.byref(g), C.byref(pp), C.byref(pp), None, None, C.byref(cfg), C.byref(pp), C.byref(pp),
             C.byref(pp), -1, C.byref(n_out), None, ws, 256, None) == INVALID          # negative capacity
    assert B._lib.tgs_accumulate_screen_grad(None, 10, None, None) == INVALID


def test_geo_stride_checks(B):
    """A geo_stride that is not 0 or a multiple of 4 of at least 12 is refused
    before any device work, in tgs_gaussians and in tgs_param_ptrs."""
    cam = B.camera(dict(viewmat=[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 4, 0, 0, 0, 1], fx=100, fy=100, cx=32, cy=32,
                        width=64, height=64))
    proj = B.Projected(P16, P16, P16, P16, P16)
    for bad in (3, 8, 13, -16):
        g = B.Gaussians(P16, P16, P16, P16, P16, 10, 3, bad)
        assert B._lib.tgs_project_gaussians(C.byref(g), C.byref(cam), None, C.byref(proj), None) == INVALID
        pp = B.ParamPtrs(P16, P16, P16, P16, P16, bad)
        ok = B.ParamPtrs(P16, P16, P16, P16, P16, 16)
        opt = B.Opt((C.c_float * 6)(*[1e-3] * 6), 0.9, 0.999, 1e-15, 1e-8, 1)
        ws = (C.c_uint8 * 1024)()       # enough for 10 Gaussians: only the stride is wrong
        assert B._lib.tgs_hybrid_step_workspace_size(10) <= 1024
        for args in ((pp, ok, ok, ok), (ok, pp, ok, ok), (ok, ok, pp, ok), (ok, ok, ok, pp)):
            assert B._lib.tgs_hybrid_step(*[C.byref(a) for a in args], 10, None, None, 0, 1, None, C.byref(opt),
                                          ws, 1024, None) == INVALID

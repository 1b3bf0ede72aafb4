"""Double-precision CPU oracle for the TurboGS sparse-sampled path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` leg of ``bench.py`` may import this
package.  The CUDA library never imports it, and the two share no code.

The arithmetic lives in ``turbogs_oracle.c`` (plain C, double precision, each
function citing the passage of TurboGS it restates); this module compiles it
with gcc on first use and marshals numpy arrays in and out with ctypes.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "turbogs_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

# loss constants (readings of Sec. 3.7 / App. A, shared with the library as values)
EPS_CHARBONNIER = 1e-3
EPS_NCC = 1e-8
BETA_EMA = 0.4


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liborc.so`` (host architecture)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_LIB)
            _declare(_lib)
    return _lib


_p = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int
_u64 = C.c_uint64
_u32 = C.c_uint32
_d = C.c_double


def _declare(L):
    L.orc_half_to_double.argtypes = [C.c_uint16]
    L.orc_half_to_double.restype = _d
    L.orc_double_to_half.argtypes = [_d]
    L.orc_double_to_half.restype = C.c_uint16
    L.orc_sh_basis.argtypes = [_p, _p, _p]
    L.orc_sh_basis.restype = None
    L.orc_project.argtypes = [_i64, _p, _p, _p, _p, _p, _i32, _p, _i32, _i32, _p, _p, _p, _p, _p, _p, _p, _p]
    L.orc_project.restype = _i32
    L.orc_bin_tiles.argtypes = [_i64, _p, _p, _p, _i32, _i32, _p, _i64, _p, _p, _p]
    L.orc_bin_tiles.restype = _i64
    L.orc_mix64.argtypes = [_u64]
    L.orc_mix64.restype = _u64
    L.orc_hash.argtypes = [_u64, _u64, _u32, _u32, _u32, _u32]
    L.orc_hash.restype = _u64
    L.orc_neglog2_q32.argtypes = [_u64]
    L.orc_neglog2_q32.restype = _u64
    L.orc_hard_key.argtypes = [_u64, _u64]
    L.orc_hard_key.restype = _d
    L.orc_err_weight.argtypes = [C.c_uint16]
    L.orc_err_weight.restype = _u64
    L.orc_choose_items.argtypes = [_i32, _p, _p, _i32, _i32, _i32, _u64, _u64, _u32, _u32, _p]
    L.orc_choose_items.restype = _i32
    L.orc_select.argtypes = [_i32, _i32, _p, _p, _i32, _i32, _i32, _i32, _i32, _i32, _u64, _u64, _u32,
                             _p, _p, _p, _p, _p]
    L.orc_select.restype = _i32
    L.orc_render_pixels.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _i32, _i32, _p, _i64, _p, _p, _p, _p,
                                    _p, _p]
    L.orc_render_pixels.restype = _i32
    L.orc_render_backward.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _i32, _i32, _p, _i64, _p, _p, _p]
    L.orc_render_backward.restype = _i32
    L.orc_error_stats.argtypes = [_i64, _p, _p, _p, _p, _p, _i32, _i32, _i64, _p, _p, _p]
    L.orc_error_stats.restype = _i32
    L.orc_project_backward.argtypes = [_i64, _p, _p, _p, _p, _p, _i32, _p, _i32, _i32, _p, _p, _p]
    L.orc_project_backward.restype = _i32
    L.orc_loss.argtypes = [_i32, _i32, _i32, _p, _p, _p, _p, _p, _p, _d, _d, _d, _p, _p, _p, _p, _p, _p]
    L.orc_loss.restype = _i32
    L.orc_loss_ssim.argtypes = [_i32, _i32, _i32, _p, _p, _p, _p, _p, _p, _d, _d, _p, _p, _p, _p, _p, _p]
    L.orc_loss_ssim.restype = _i32
    L.orc_cholesky_solve.argtypes = [_p, _p, _p, _i32]
    L.orc_cholesky_solve.restype = _i32
    L.orc_hybrid_step.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _i32, _i32, _i32, _p]
    L.orc_hybrid_step.restype = _i32
    L.orc_round_bf16.argtypes = [_d]
    L.orc_round_bf16.restype = _d
    L.orc_mlp_forward.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _p, _i32, _p, _p, _p]
    L.orc_mlp_forward.restype = _i32
    L.orc_mlp_backward.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _p, _p, _i32, _p, _p, _p, _p, _p, _p, _p]
    L.orc_mlp_backward.restype = _i32
    L.orc_tile_observe.argtypes = [_i32, _p, _p, _p, _p, _p, _i64, _p, _p, _p, _i32]
    L.orc_tile_observe.restype = None
    L.orc_tile_features.argtypes = [_i32, _p, _p, _p, _i32, _d, _d, _d, _d, _d, _i64, _p]
    L.orc_tile_features.restype = None
    L.orc_tile_refresh.argtypes = [_p, _p, _p, _i32, _i32]
    L.orc_tile_refresh.restype = None
    L.orc_view_error_sums.argtypes = [_p, _i32, _i64, _i32, _i32, _p]
    L.orc_view_error_sums.restype = None
    L.orc_log2_q32.argtypes = [_u64]
    L.orc_log2_q32.restype = _u64
    L.orc_view_pose.argtypes = [_p, _p, _p]
    L.orc_view_pose.restype = None
    L.orc_sample_views.argtypes = [_p, _p, _i32, _i32, _d, _d, _u64, _u64, _p, _p]
    L.orc_sample_views.restype = None
    L.orc_accumulate_screen_grad.argtypes = [_i64, _p, _p]
    L.orc_accumulate_screen_grad.restype = None
    L.orc_density_control.argtypes = [_i64, _p, _p, _p, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float,
                                      _i32, _i32, _i32, _i64, _p, _p, _p]
    L.orc_density_control.restype = _i64
    L.orc_gaussian_scores.argtypes = [_i64, _p, _i32, _d, _d, _d, _p, _p]
    L.orc_gaussian_scores.restype = None


def _c(a, dtype):
    """Contiguous copy/view of ``a`` with ``dtype``; None stays None."""
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data


def camera_array(cam) -> np.ndarray:
    """[viewmat 16 (row-major world->camera), fx, fy, cx, cy, znear] in float64."""
    v = np.asarray(cam["viewmat"], dtype=np.float64).reshape(16)
    return np.concatenate([v, np.array([cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["znear"]],
                                       dtype=np.float64)])


# ----------------------------------------------------------------------------
# wrappers
# ----------------------------------------------------------------------------

def half_to_double(h: int) -> float:
    return lib().orc_half_to_double(int(h))


def double_to_half(x: float) -> int:
    return int(lib().orc_double_to_half(float(x)))


def sh_basis(d):
    """Real SH basis (16) and its polynomial gradient (16, 3) at unit direction d."""
    d = _c(d, np.float64)
    Y = np.zeros(16)
    G = np.zeros(48)
    lib().orc_sh_basis(_ptr(d), _ptr(Y), _ptr(G))
    return Y, G.reshape(16, 3)


def project(g, cam, sh_degree=3, tile_rank=None):
    """Project Gaussians (dict of means, log_scales, quats, opacity_logits, sh)."""
    n = int(np.asarray(g["means"]).shape[0])
    means = _c(g["means"], np.float64)
    ls = _c(g["log_scales"], np.float64)
    q = _c(g["quats"], np.float64)
    ol = _c(g["opacity_logits"], np.float64)
    sh = _c(np.asarray(g["sh"]).reshape(n, 48), np.float64)
    camv = camera_array(cam)
    tr = _c(tile_rank, np.int32)
    out = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), opac=np.zeros(n), rgb=np.zeros((n, 3)),
               depth=np.zeros(n), radius=np.zeros(n, np.int32), margin=np.zeros(n))
    lib().orc_project(n, _ptr(means), _ptr(ls), _ptr(q), _ptr(ol), _ptr(sh), int(sh_degree), _ptr(camv),
                      int(cam["width"]), int(cam["height"]), _ptr(tr), _ptr(out["xy"]), _ptr(out["conic"]),
                      _ptr(out["opac"]), _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["radius"]),
                      _ptr(out["margin"]))
    return out


def bin_tiles(xy, radius, depth, width, height, tile_rank=None, capacity=None):
    """Sorted (key, Gaussian id) pairs of every (active tile, Gaussian) overlap."""
    xy = _c(xy, np.float32)
    radius = _c(radius, np.int32)
    depth = _c(depth, np.float32)
    n = radius.shape[0]
    tiles = ((width + 15) // 16) * ((height + 15) // 16)
    tr = _c(tile_rank, np.int32)
    counts = np.zeros(tiles, np.int32)
    if capacity is None:
        dummy = np.zeros(1, np.uint64)
        capacity = int(lib().orc_bin_tiles(n, _ptr(xy), _ptr(radius), _ptr(depth), width, height, _ptr(tr), -1,
                                           _ptr(dummy), _ptr(dummy), _ptr(counts)))
    keys = np.zeros(max(capacity, 1), np.uint64)
    vals = np.zeros(max(capacity, 1), np.int32)
    total = lib().orc_bin_tiles(n, _ptr(xy), _ptr(radius), _ptr(depth), width, height, _ptr(tr), capacity,
                                _ptr(keys), _ptr(vals), _ptr(counts))
    if total < 0:
        return None
    return keys[:total], vals[:total], counts


def mix64(z: int) -> int:
    return int(lib().orc_mix64(z & (2**64 - 1)))


def hash_(seed, it, view, stream, tile, item) -> int:
    return int(lib().orc_hash(seed, it, view, stream, tile, item))


def neglog2_q32(h: int) -> int:
    return int(lib().orc_neglog2_q32(h & (2**64 - 1)))


def hard_key(w: int, L: int) -> float:
    return float(lib().orc_hard_key(int(w), int(L)))


def err_weight(h: int) -> int:
    return int(lib().orc_err_weight(int(h)))


def choose_items(w, age, n, hard_pm=400, stable_pm=300, seed=0, it=0, view=0, tile=0):
    w = _c(w, np.uint64)
    age = _c(age, np.uint32)
    cnt = w.shape[0]
    out = np.zeros(cnt, np.uint8)
    lib().orc_choose_items(cnt, _ptr(w), _ptr(age), int(n), hard_pm, stable_pm, seed, it, view, tile, _ptr(out))
    return out.astype(bool)


def select(err_f16_bits, age, width, height, n_select, n_pix, tile_hard_pm=400, tile_stable_pm=300,
           pix_hard_pm=400, pix_stable_pm=300, seed=0, it=0, view=0):
    err = _c(err_f16_bits, np.uint16)
    age = _c(age, np.uint16)
    tiles = ((width + 15) // 16) * ((height + 15) // 16)
    active = np.zeros(tiles, np.int32)
    n_active = np.zeros(1, np.int32)
    rank = np.zeros(tiles, np.int32)
    off = np.zeros(tiles + 1, np.int32)
    idx = np.zeros(tiles * 256, np.uint8)
    lib().orc_select(width, height, _ptr(err), _ptr(age), int(n_select), int(n_pix), tile_hard_pm,
                     tile_stable_pm, pix_hard_pm, pix_stable_pm, seed, it, view, _ptr(active), _ptr(n_active),
                     _ptr(rank), _ptr(off), _ptr(idx))
    A = int(n_active[0])
    return dict(active_tiles=active[:A], n_active=A, tile_rank=rank, pix_off=off[:A + 1],
                pix_idx=idx[:off[A]])


def pixel_coords(active_tiles, pix_off, pix_idx, width):
    """Integer pixel coordinates [P,2] of a sampled set (tile order)."""
    tx_n = (width + 15) // 16
    counts = np.diff(np.asarray(pix_off))
    tiles = np.repeat(np.asarray(active_tiles), counts)
    l = np.asarray(pix_idx).astype(np.int32)
    x = (tiles % tx_n) * 16 + (l % 16)
    y = (tiles // tx_n) * 16 + (l // 16)
    return np.stack([x, y], 1).astype(np.int32)


def render_pixels(proj, width, height, pix_xy, bg=(0.0, 0.0, 0.0)):
    xy = _c(proj["xy"], np.float64)
    conic = _c(proj["conic"], np.float64)
    opac = _c(proj["opac"], np.float64)
    rgb = _c(proj["rgb"], np.float64)
    depth = _c(proj["depth"], np.float64)
    radius = _c(proj["radius"], np.int32)
    n = radius.shape[0]
    pix = _c(pix_xy, np.int32).reshape(-1, 2)
    P = pix.shape[0]
    bgv = _c(bg, np.float64)
    out = dict(rgb=np.zeros((P, 3)), T=np.zeros(P), n_last=np.zeros(P, np.int32),
               n_contrib=np.zeros(P, np.int32), margin=np.zeros(P))
    lib().orc_render_pixels(n, _ptr(xy), _ptr(conic), _ptr(opac), _ptr(rgb), _ptr(depth), _ptr(radius),
                            width, height, _ptr(bgv), P, _ptr(pix), _ptr(out["rgb"]), _ptr(out["T"]),
                            _ptr(out["n_last"]), _ptr(out["n_contrib"]), _ptr(out["margin"]))
    return out


def render_backward(proj, width, height, pix_xy, dL_drgb, bg=(0.0, 0.0, 0.0)):
    """grad2d [N,9] = (dx, dy, da, db, dc, dopacity, dr, dg, db)."""
    xy = _c(proj["xy"], np.float64)
    conic = _c(proj["conic"], np.float64)
    opac = _c(proj["opac"], np.float64)
    rgb = _c(proj["rgb"], np.float64)
    depth = _c(proj["depth"], np.float64)
    radius = _c(proj["radius"], np.int32)
    n = radius.shape[0]
    pix = _c(pix_xy, np.int32).reshape(-1, 2)
    g = _c(dL_drgb, np.float64).reshape(-1, 3)
    bgv = _c(bg, np.float64)
    out = np.zeros((n, 9))
    lib().orc_render_backward(n, _ptr(xy), _ptr(conic), _ptr(opac), _ptr(rgb), _ptr(depth), _ptr(radius),
                              width, height, _ptr(bgv), pix.shape[0], _ptr(pix), _ptr(g), _ptr(out))
    return out


def error_stats(proj, width, height, pix_xy, err):
    """Sec. 3.8, Eq. 12 over the listed pixels: stats [N,3] =
    (sum e w, sum w, sum D w) with w = T alpha the compositing weight and D the
    conic Mahalanobis distance of the pixel centre from the splat."""
    xy = _c(proj["xy"], np.float64)
    conic = _c(proj["conic"], np.float64)
    opac = _c(proj["opac"], np.float64)
    depth = _c(proj["depth"], np.float64)
    radius = _c(proj["radius"], np.int32)
    n = radius.shape[0]
    pix = _c(pix_xy, np.int32).reshape(-1, 2)
    e = _c(err, np.float64).reshape(-1)
    out = np.zeros((n, 3))
    lib().orc_error_stats(n, _ptr(xy), _ptr(conic), _ptr(opac), _ptr(depth), _ptr(radius), width, height,
                          pix.shape[0], _ptr(pix), _ptr(e), _ptr(out))
    return out


def project_backward(g, cam, grad2d, sh_degree=3, tile_rank=None):
    """grads [N,59] = (means 3, log_scales 3, quats 4, opacity logit 1, sh 48)."""
    n = int(np.asarray(g["means"]).shape[0])
    means = _c(g["means"], np.float64)
    ls = _c(g["log_scales"], np.float64)
    q = _c(g["quats"], np.float64)
    ol = _c(g["opacity_logits"], np.float64)
    sh = _c(np.asarray(g["sh"]).reshape(n, 48), np.float64)
    camv = camera_array(cam)
    tr = _c(tile_rank, np.int32)
    g2 = _c(grad2d, np.float64)
    out = np.zeros((n, 59))
    lib().orc_project_backward(n, _ptr(means), _ptr(ls), _ptr(q), _ptr(ol), _ptr(sh), int(sh_degree),
                               _ptr(camv), int(cam["width"]), int(cam["height"]), _ptr(tr), _ptr(g2), _ptr(out))
    return out


def loss(width, height, sel, rgb, target, err_f16_bits=None, age=None, lambda_in=None,
         eps_c=EPS_CHARBONNIER, eps_n=EPS_NCC, beta=BETA_EMA):
    """Fused sparse loss.  Returns dict; error/age maps are updated copies."""
    active = _c(sel["active_tiles"], np.int32)
    off = _c(sel["pix_off"], np.int32)
    idx = _c(sel["pix_idx"], np.uint8)
    A = int(active.shape[0])
    P = int(off[A])
    rgb = _c(rgb, np.float64).reshape(-1, 3)
    tgt = _c(target, np.float64)
    err = None if err_f16_bits is None else np.array(err_f16_bits, dtype=np.uint16, copy=True)
    ag = None if age is None else np.array(age, dtype=np.uint16, copy=True)
    lam_in = _c(lambda_in, np.float64)
    out = dict(dL_drgb=np.zeros((P, 3)), lam=np.zeros(max(A, 1)), err=np.zeros(max(P, 1)),
               loss=np.zeros(1))
    lib().orc_loss(width, height, A, _ptr(active), _ptr(off), _ptr(idx if idx.size else np.zeros(1, np.uint8)),
                   _ptr(rgb), _ptr(tgt), _ptr(lam_in), eps_c, eps_n, beta, _ptr(err), _ptr(ag),
                   _ptr(out["dL_drgb"]), _ptr(out["lam"]), _ptr(out["err"]), _ptr(out["loss"]))
    out["lam"] = out["lam"][:A]
    out["err"] = out["err"][:P]
    out["loss"] = float(out["loss"][0])
    out["err_map"] = err
    out["age_map"] = ag
    return out


def loss_ssim(width, height, sel, rgb, target, err_f16_bits=None, age=None, lambda_in=None,
              eps_c=EPS_CHARBONNIER, beta=BETA_EMA):
    """The sparse loss with the SSIM structure term (Table 4's S-SSIM
    variant); arguments and outputs as ``loss``."""
    active = _c(sel["active_tiles"], np.int32)
    off = _c(sel["pix_off"], np.int32)
    idx = _c(sel["pix_idx"], np.uint8)
    A = int(active.shape[0])
    P = int(off[A])
    rgb = _c(rgb, np.float64).reshape(-1, 3)
    tgt = _c(target, np.float64)
    err = None if err_f16_bits is None else np.array(err_f16_bits, dtype=np.uint16, copy=True)
    ag = None if age is None else np.array(age, dtype=np.uint16, copy=True)
    lam_in = _c(lambda_in, np.float64)
    out = dict(dL_drgb=np.zeros((P, 3)), lam=np.zeros(max(A, 1)), err=np.zeros(max(P, 1)), loss=np.zeros(1))
    lib().orc_loss_ssim(width, height, A, _ptr(active), _ptr(off),
                        _ptr(idx if idx.size else np.zeros(1, np.uint8)), _ptr(rgb), _ptr(tgt), _ptr(lam_in),
                        eps_c, beta, _ptr(err), _ptr(ag), _ptr(out["dL_drgb"]), _ptr(out["lam"]), _ptr(out["err"]),
                        _ptr(out["loss"]))
    out["lam"] = out["lam"][:A]
    out["err"] = out["err"][:P]
    out["loss"] = float(out["loss"][0])
    out["err_map"] = err
    out["age_map"] = ag
    return out


def cholesky_solve(A, b):
    A = _c(A, np.float64)
    b = _c(b, np.float64)
    x = np.zeros_like(b)
    rc = lib().orc_cholesky_solve(_ptr(A), _ptr(b), _ptr(x), b.shape[0])
    if rc != 0:
        raise np.linalg.LinAlgError("not positive definite")
    return x


def hybrid_step(params, grads, m, v, touched, step, mode, cfg, rows=None):
    """One hybrid step on packed [N,59] rows (copies in, updated copies out)."""
    p = np.array(params, dtype=np.float64, copy=True)
    mm = np.array(m, dtype=np.float64, copy=True)
    vv = np.array(v, dtype=np.float64, copy=True)
    g = _c(grads, np.float64)
    t = _c(touched, np.uint8)
    r = _c(rows, np.float64)
    k = 0 if rows is None else int(np.asarray(rows).shape[0])
    c = _c(cfg, np.float64)
    lib().orc_hybrid_step(p.shape[0], _ptr(p), _ptr(g), _ptr(mm), _ptr(vv), _ptr(t), _ptr(r), k, int(step),
                          int(mode), _ptr(c))
    return p, mm, vv


# ----------------------------------------------------------------------------
# tile-error predictor (MLP 16 -> 128 -> 128 -> 1)
# ----------------------------------------------------------------------------

def round_bf16(x: float) -> float:
    return float(lib().orc_round_bf16(float(x)))


def _mlp_w(w):
    return [_c(w[k], np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]


def mlp_forward(x, w, bf16=True):
    """y [R], h1 [R,128], h2 [R,128] for features x [R,16]."""
    x = _c(x, np.float64).reshape(-1, 16)
    R = x.shape[0]
    W1, b1, W2, b2, W3, b3 = _mlp_w(w)
    y, h1, h2 = np.zeros(R), np.zeros((R, 128)), np.zeros((R, 128))
    lib().orc_mlp_forward(R, _ptr(x), _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2), _ptr(W3), _ptr(b3), int(bf16),
                          _ptr(y), _ptr(h1), _ptr(h2))
    return y, h1, h2


def mlp_backward(x, t, w, bf16=True):
    """loss and gradient dict (W1, b1, W2, b2, W3, b3) of mean (y - t)^2 / 2."""
    x = _c(x, np.float64).reshape(-1, 16)
    t = _c(t, np.float64)
    R = x.shape[0]
    W1, b1, W2, b2, W3, b3 = _mlp_w(w)
    g = dict(W1=np.zeros((128, 16)), b1=np.zeros(128), W2=np.zeros((128, 128)), b2=np.zeros(128),
             W3=np.zeros(128), b3=np.zeros(1))
    loss = np.zeros(1)
    lib().orc_mlp_backward(R, _ptr(x), _ptr(t), _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2), _ptr(W3), _ptr(b3),
                           int(bf16), _ptr(loss), _ptr(g["W1"]), _ptr(g["b1"]), _ptr(g["W2"]), _ptr(g["b2"]),
                           _ptr(g["W3"]), _ptr(g["b3"]))
    return float(loss[0]), g


# ----------------------------------------------------------------------------
# tile memory, features and refresh (tile-error predictor)
# ----------------------------------------------------------------------------

def tile_observe(n_active, active_tiles, pix_off, ranges, T_final, err_pix, iter_, mem, mem_iter, residual=False):
    """Updates mem [T,4] (float64) and mem_iter [T] (int64) in place; returns
    the targets [n_active]."""
    L = lib()
    at, po = _c(active_tiles, np.int32), _c(pix_off, np.int32)
    rg = _c(ranges, np.int32)
    Tf, ep = _c(T_final, np.float64), _c(err_pix, np.float64)
    assert mem.dtype == np.float64 and mem.flags.c_contiguous and mem_iter.dtype == np.int64
    tgt = np.zeros(max(int(n_active), 1))
    L.orc_tile_observe(int(n_active), _ptr(at), _ptr(po), _ptr(rg), _ptr(Tf), _ptr(ep), int(iter_), _ptr(mem),
                       _ptr(mem_iter), _ptr(tgt), 1 if residual else 0)
    return tgt[:int(n_active)]


def tile_features(mem, mem_iter, cam, rows=None, n_rows=None, view_cos=1.0, iter_=0):
    L = lib()
    W = int(cam["width"])
    r = _c(rows, np.int32)
    n = int(n_rows if n_rows is not None else (len(rows) if rows is not None else mem.shape[0]))
    x = np.zeros((max(n, 1), 16))
    L.orc_tile_features(n, _ptr(r), _ptr(_c(mem, np.float64)), _ptr(_c(mem_iter, np.int64)), W, float(cam["fx"]),
                        float(cam["fy"]), float(cam["cx"]), float(cam["cy"]), float(view_cos), int(iter_), _ptr(x))
    return x[:n]


def tile_refresh(pred, err_f16_bits, width, height, base=None):
    """Returns the refreshed error map (uint16 fp16 bit patterns)."""
    L = lib()
    e = np.array(err_f16_bits, dtype=np.uint16, copy=True, order="C")
    L.orc_tile_refresh(_ptr(_c(pred, np.float64)), _ptr(_c(base, np.float64)), _ptr(e), int(width), int(height))
    return e


# ----------------------------------------------------------------------------
# view sampling and its schedule (Sec. 3.4; App. A)
# ----------------------------------------------------------------------------

def view_error_sums(maps_f16_bits) -> np.ndarray:
    """Per view, the exact sum of E * 2^24 over its pixels (Eq. 5 times
    W H 2^24).  maps [V,H,W] fp16 bit patterns."""
    m = _c(maps_f16_bits, np.uint16)
    V, H, W = m.shape
    out = np.zeros(V, np.uint64)
    lib().orc_view_error_sums(_ptr(m), V, H * W, W, H, _ptr(out))
    return out


def log2_q32(x: int) -> int:
    return int(lib().orc_log2_q32(int(x)))


def view_pose(viewmat):
    """(centre, unit forward axis) of a row-major world-to-camera matrix."""
    v = _c(np.asarray(viewmat).reshape(16), np.float32)
    c, d = np.zeros(3), np.zeros(3)
    lib().orc_view_pose(_ptr(v), _ptr(c), _ptr(d))
    return c, d


def sample_views(sums, viewmats, k, lambda_d, lambda_theta, seed=0, it=0, stack=None):
    """One geometry-aware draw (Eqs. 5-6).  Returns (views [k]: anchor first,
    then the draws ascending; the updated stack [V] uint8)."""
    s = _c(sums, np.uint64)
    vm = _c(np.asarray(viewmats).reshape(-1, 16), np.float32)
    V = s.shape[0]
    st = np.ones(V, np.uint8) if stack is None else np.array(stack, dtype=np.uint8, copy=True, order="C")
    out = np.zeros(k, np.int32)
    lib().orc_sample_views(_ptr(s), _ptr(vm), V, int(k), float(lambda_d), float(lambda_theta), int(seed), int(it),
                           _ptr(st), _ptr(out))
    return out, st


def sampling_schedule(t, E_t, E_init, K_max=10, K_min=3, alpha=3.0, tau_until=3500, lam=1.0, eps=1e-8):
    """(K_t, r_tile) of the adaptive schedule (App. A, Eqs. 15-16).

    r = clip(E_t / (E_init + eps), 0, 1), phi = sin(pi/2 sqrt(r)),
    rho = 1 - clip(t / tau_until, 0, 1) (the appendix's definition, 1 at the
    start and 0 from tau_until on), g = 1 - rho phi;
    r_tile = r_min + (r_max - r_min) g with r_min = lam / K_max and
    r_max = lam / K_min; K_t = round(K_min + (K_max - K_min) exp(-alpha g)),
    rounding halves up."""
    r = min(max(E_t / (E_init + eps), 0.0), 1.0)
    phi = math.sin(0.5 * math.pi * math.sqrt(r))
    rho = 1.0 - min(max(t / tau_until, 0.0), 1.0)
    g = 1.0 - rho * phi
    r_min, r_max = lam / K_max, lam / K_min
    r_tile = r_min + (r_max - r_min) * g
    K = int(math.floor(K_min + (K_max - K_min) * math.exp(-alpha * g) + 0.5))
    return K, r_tile


# ----------------------------------------------------------------------------
# density control scores (Sec. 3.8)
# ----------------------------------------------------------------------------

def gaussian_scores(stats, t, tau_until=3500, lambda_base=0.8, eps=1e-8):
    """(e [N], s [N]) of Eq. 13 from statistics rows (E, W, D, ...) of
    Eq. 12 at iteration t; the progress rho = min(1, t / tau_until)."""
    st = _c(stats, np.float64)
    n, stride = st.shape
    e, s = np.zeros(n), np.zeros(n)
    rho = min(1.0, max(0.0, t / tau_until))
    lib().orc_gaussian_scores(n, _ptr(st), stride, float(lambda_base), rho, float(eps), _ptr(e), _ptr(s))
    return e, s


def accumulate_screen_grad(grad2d, accum):
    """accum [N,2] float32 (updated in place) += (|(dx, dy)|, 1) where the
    view's grad2d [N,12] row is not all zero."""
    g = _c(grad2d, np.float32)
    assert accum.dtype == np.float32 and accum.flags.c_contiguous
    lib().orc_accumulate_screen_grad(g.shape[0], _ptr(g), _ptr(accum))
    return accum


def density_control(params, stats, accum, lam_eff, tau_grad, log_split, logit_prune, topk_pm=800, final=False,
                    final_pm=900, eps=1e-8):
    """One density-control step (Sec. 3.8, Eq. 13; the procedure's reading in
    the C source).  params: packed [N,59] float32 rows.  Returns (out [M,59]
    float64, src [M] input index, kind [M]: 0 kept, 1 clone copy, 2/3 split
    children)."""
    p = _c(params, np.float32)
    st = _c(stats, np.float32)
    ac = _c(accum, np.float32)
    n = p.shape[0]
    cap = 2 * max(n, 1)
    out = np.zeros((cap, 59))
    src = np.zeros(cap, np.int64)
    kind = np.zeros(cap, np.int32)
    m = lib().orc_density_control(n, _ptr(p), _ptr(st), _ptr(ac), float(lam_eff), float(eps), float(tau_grad),
                                  float(log_split), float(logit_prune), int(topk_pm), 1 if final else 0,
                                  int(final_pm), cap, _ptr(out), _ptr(src), _ptr(kind))
    return out[:m], src[:m], kind[:m]

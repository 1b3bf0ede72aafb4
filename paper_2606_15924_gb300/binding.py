"""Python binding of the C ABI in include/turbogs.h (argument marshalling only).

Every function here has the name of the C entry point without its ``tgs_``
prefix, takes torch CUDA tensors (contiguous, of the dtype and shape the header
states) and launches on the current torch stream unless one is given.  All the
arithmetic runs in ``libturbogs.so``; importing this module loads it and raises
if it is missing - there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libturbogs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libturbogs.so not found at {LIB_PATH}: build it with "
                      "`python -m paper_2606_15924_gb300.build` (needs nvcc)")
_lib = C.CDLL(LIB_PATH)

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_DEVICE = range(6)


class TgsError(RuntimeError):
    def __init__(self, fn, status):
        msg = _lib.tgs_status_string(status).decode()
        if status == ERR_CUDA:
            msg += f" (cudaError {_lib.tgs_last_cuda_error()})"
        super().__init__(f"{fn}: {msg}")
        self.status = status


# ----------------------------------------------------------------------------
# structs
# ----------------------------------------------------------------------------

class Camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32), ("znear", C.c_float)]


class Gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64), ("sh_degree", C.c_int32),
                ("geo_stride", C.c_int32)]


class ParamPtrs(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("geo_stride", C.c_int32)]


class Projected(C.Structure):
    _fields_ = [("xy", C.c_void_p), ("conic_opac", C.c_void_p), ("rgb", C.c_void_p), ("depth", C.c_void_p),
                ("radius", C.c_void_p)]


class Sampling(C.Structure):
    _fields_ = [("tile_hard_pm", C.c_int32), ("tile_stable_pm", C.c_int32), ("pix_hard_pm", C.c_int32),
                ("pix_stable_pm", C.c_int32)]


class LossParams(C.Structure):
    _fields_ = [("eps_charbonnier", C.c_float), ("eps_ncc", C.c_float), ("beta", C.c_float),
                ("view_weight", C.c_float)]


class DensityParams(C.Structure):
    _fields_ = [("lambda_eff", C.c_float), ("eps", C.c_float), ("tau_grad", C.c_float),
                ("log_scale_split", C.c_float), ("opacity_logit_prune", C.c_float), ("topk_permille", C.c_int32),
                ("final_prune", C.c_int32), ("final_permille", C.c_int32)]


class Mlp(C.Structure):
    _fields_ = [("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p), ("w3", C.c_void_p),
                ("b3", C.c_void_p)]


class Checkpoints(C.Structure):
    _fields_ = [("data", C.c_void_p), ("n_slots", C.c_int32), ("stride", C.c_int64), ("rgb", C.c_void_p),
                ("tile_last", C.c_void_p)]


class ViewBatch(C.Structure):
    _fields_ = [("proj", Projected), ("tile_ranges", C.c_void_p), ("vals", C.c_void_p),
                ("active_tiles", C.c_void_p), ("n_active", C.c_void_p), ("n_active_max", C.c_int32),
                ("pix_off", C.c_void_p), ("pix_idx", C.c_void_p), ("n_pix_max", C.c_int32), ("cam", Camera),
                ("bg", C.c_float * 3), ("rgb", C.c_void_p), ("T_final", C.c_void_p), ("n_last", C.c_void_p),
                ("dL_drgb", C.c_void_p), ("grad2d", C.c_void_p), ("n_gaussians", C.c_int64),
                ("ckpt", Checkpoints)]


class Opt(C.Structure):
    _fields_ = [("lr", C.c_float * 6), ("beta1", C.c_float), ("beta2", C.c_float), ("eps_adam", C.c_float),
                ("eps_lm", C.c_float), ("mode", C.c_int32)]


_p = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_u64 = C.c_uint64
_u32 = C.c_uint32
_sz = C.c_size_t
_P = C.POINTER

_lib.tgs_version.restype = C.c_char_p
_lib.tgs_status_string.restype = C.c_char_p
_lib.tgs_status_string.argtypes = [_i32]
_lib.tgs_last_cuda_error.restype = _i32
_lib.tgs_device_check.restype = _i32
_lib.tgs_graph_count_kernels.restype = _i64
_lib.tgs_graph_count_kernels.argtypes = [_p]
_lib.tgs_advance_counters.restype = _i32
_lib.tgs_advance_counters.argtypes = [_p, _p, _p]
_lib.tgs_select_tiles_workspace_size.restype = _sz
_lib.tgs_select_tiles_workspace_size.argtypes = [_i32, _i32]
_lib.tgs_select_tiles.restype = _i32
_lib.tgs_select_tiles.argtypes = [_p, _p, _i32, _i32, _i32, _i32, _P(Sampling), _u64, _u64, _p, _u32, _p, _sz,
                                  _p, _p, _p, _p, _p, _p]
_lib.tgs_select_tiles_noalloc.restype = _i32
_lib.tgs_select_tiles_noalloc.argtypes = [_p, _p, _i32, _i32, _i32, _i32, _P(Sampling), _u64, _u64, _p, _u32,
                                          _p, _p, _p, _p, _p, _p]
_lib.tgs_project_gaussians.restype = _i32
_lib.tgs_project_gaussians.argtypes = [_P(Gaussians), _P(Camera), _p, _P(Projected), _p]
_lib.tgs_bin_tiles_workspace_size.restype = _sz
_lib.tgs_bin_tiles_workspace_size.argtypes = [_i64, _i64, _i32]
_lib.tgs_bin_tiles.restype = _i32
_lib.tgs_bin_tiles.argtypes = [_P(Projected), _i64, _P(Camera), _p, _i32, _p, _sz, _i64, _p, _p, _p, _p, _p]
_lib.tgs_render_sampled.restype = _i32
_lib.tgs_checkpoint_bytes.restype = _sz
_lib.tgs_checkpoint_bytes.argtypes = [_i32, _i32, _i32]
_lib.tgs_set_forward_split.restype = _i32
_lib.tgs_set_forward_split.argtypes = [_i32]
_lib.tgs_render_sampled.argtypes = [_P(Projected), _p, _p, _p, _p, _i32, _p, _p, _i32, _P(Camera), _p, _p, _p,
                                    _p, _P(Checkpoints), _p]
_lib.tgs_loss_sparse_ncc.restype = _i32
_lib.tgs_loss_sparse_ncc.argtypes = [_p, _p, _i32, _i32, _p, _p, _i32, _p, _p, _i32, _P(LossParams), _p, _p, _p,
                                     _p, _p, _p, _p]
_lib.tgs_loss_sparse_ssim.restype = _i32
_lib.tgs_loss_sparse_ssim.argtypes = [_p, _p, _i32, _i32, _p, _p, _i32, _p, _p, _i32, _P(LossParams), _p, _p, _p,
                                     _p, _p, _p, _p]
_lib.tgs_backward_sampled.restype = _i32
_lib.tgs_backward_sampled.argtypes = [_P(Gaussians), _P(Camera), _P(Projected), _p, _p, _p, _p, _i32, _p, _p,
                                      _i32, _p, _p, _p, _p, _p, _P(ParamPtrs), _p, _i32, _P(Checkpoints), _p]
_lib.tgs_render_backward_sampled.restype = _i32
_lib.tgs_error_stats_sampled.restype = _i32
_lib.tgs_error_stats_sampled.argtypes = [_P(Projected), _p, _p, _p, _p, _i32, _p, _p, _i32, _P(Camera), _p, _p, _p,
                                         _i64, _i32, _p]
_lib.tgs_render_backward_sampled.argtypes = [_P(Projected), _p, _p, _p, _p, _i32, _p, _p, _i32, _P(Camera), _p, _p,
                                             _p, _p, _p, _i64, _P(Checkpoints), _p]
_lib.tgs_render_backward_sampled_stats.restype = _i32
_lib.tgs_render_backward_sampled_stats.argtypes = [_P(Projected), _p, _p, _p, _p, _i32, _p, _p, _i32, _P(Camera), _p,
                                                   _p, _p, _p, _p, _i64, _P(Checkpoints), _p, _p, _i32, _p]
_lib.tgs_accumulate_screen_grad.restype = _i32
_lib.tgs_accumulate_screen_grad.argtypes = [_p, _i64, _p, _p]
_lib.tgs_density_control_workspace_size.restype = _sz
_lib.tgs_density_control_workspace_size.argtypes = [_i64]
_lib.tgs_density_control.restype = _i32
_lib.tgs_density_control.argtypes = [_P(Gaussians), _P(ParamPtrs), _P(ParamPtrs), _p, _p, _P(DensityParams),
                                     _P(ParamPtrs), _P(ParamPtrs), _P(ParamPtrs), _i64, _p, _p, _p, _sz, _p]
_lib.tgs_project_backward.restype = _i32
_lib.tgs_project_backward.argtypes = [_P(Gaussians), _P(Camera), _P(Projected), _p, _P(ParamPtrs), _p, _i32, _i32,
                                      _p, _p]
_lib.tgs_project_backward_multi.restype = _i32
_lib.tgs_project_backward_multi_workspace_size.restype = _sz
_lib.tgs_project_backward_multi_workspace_size.argtypes = [_i64]
_lib.tgs_project_backward_multi.argtypes = [_P(Gaussians), _i32, _P(Camera), _p, _p, _P(ParamPtrs), _p, _i32, _p,
                                            _p, _sz, _p]
_lib.tgs_project_backward_update.restype = _i32
_lib.tgs_project_backward_update.argtypes = [_P(ParamPtrs), _i64, _i32, _i32, _P(Camera), _p, _p, _P(ParamPtrs),
                                             _P(ParamPtrs), _p, _P(Opt), _i32, _p, _p, _sz, _p]
_lib.tgs_render_batched_resident.restype = _i32
_lib.tgs_render_batched_resident.argtypes = [_i32, _i32, _P(_i32)]
_lib.tgs_render_sampled_batched.restype = _i32
_lib.tgs_render_sampled_batched.argtypes = [_P(ViewBatch), _i32, _i32, _p, _p]
_lib.tgs_render_backward_batched.restype = _i32
_lib.tgs_render_backward_batched.argtypes = [_P(ViewBatch), _i32, _i32, _p, _p]
_lib.tgs_render_backward_batched_stats.restype = _i32
_lib.tgs_render_backward_batched_stats.argtypes = [_P(ViewBatch), _i32, _i32, _p, _P(_p), _p, _i64, _i32, _p]
_lib.tgs_hybrid_step.restype = _i32
_lib.tgs_hybrid_step_workspace_size.restype = _sz
_lib.tgs_hybrid_step_workspace_size.argtypes = [_i64]
_lib.tgs_hybrid_step.argtypes = [_P(ParamPtrs), _P(ParamPtrs), _P(ParamPtrs), _P(ParamPtrs), _i64, _p, _p, _i32,
                                 _i32, _p, _P(Opt), _p, _sz, _p]

_lib.tgs_mlp_param_count.restype = _i32
_lib.tgs_mlp_forward.restype = _i32
_lib.tgs_mlp_forward.argtypes = [_P(Mlp), _i64, _p, _p, _p, _p, _p]
_lib.tgs_mlp_forward_tc.restype = _i32
_lib.tgs_mlp_forward_tc.argtypes = [_P(Mlp), _i64, _p, _p, _p, _p, _p, _p]
_lib.tgs_mlp_tc_wait_drill.restype = _i32
_lib.tgs_mlp_tc_wait_drill.argtypes = [_p, _p]
_lib.tgs_mlp_backward_workspace_size.restype = _sz
_lib.tgs_mlp_backward_workspace_size.argtypes = [_i64]
_lib.tgs_mlp_backward.restype = _i32
_lib.tgs_mlp_backward.argtypes = [_P(Mlp), _i64, _p, _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p]
_lib.tgs_mlp_backward_tc.restype = _i32
_lib.tgs_mlp_backward_tc.argtypes = [_P(Mlp), _i64, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p]
_lib.tgs_mlp_train_tc.restype = _i32
_lib.tgs_mlp_train_tc.argtypes = [_P(Mlp), _i64, _p, _p, _p, _p, _p, _p, _p, _p]
_lib.tgs_tile_observe.restype = _i32
_lib.tgs_tile_observe.argtypes = [_p, _p, _i32, _p, _p, _p, _p, _u64, _p, _p, _p, _p, _i32, _p]
_lib.tgs_tile_features.restype = _i32
_lib.tgs_tile_features.argtypes = [_p, _p, _p, _p, _i32, _P(Camera), C.c_float, _u64, _p, _p, _p]
_lib.tgs_tile_refresh.restype = _i32
_lib.tgs_tile_refresh.argtypes = [_p, _p, _p, _i32, _i32, _p]
_lib.tgs_view_error_sums.restype = _i32
_lib.tgs_view_error_sums.argtypes = [_p, _i32, _i64, _i32, _i32, _p, _p]
_lib.tgs_sample_views.restype = _i32
_lib.tgs_sample_views.argtypes = [_p, _p, _i32, _i32, C.c_double, C.c_double, _u64, _u64, _p, _p, _p]
_lib.tgs_mlp_adam.restype = _i32
_lib.tgs_mlp_adam.argtypes = [_p, _p, _p, _p, _i32, C.c_float, C.c_float, C.c_float, C.c_float, _p, _p, _p, _p]

EXPORTED = ["tgs_version", "tgs_last_cuda_error", "tgs_status_string", "tgs_device_check", "tgs_graph_count_kernels",
            "tgs_advance_counters",
            "tgs_select_tiles_workspace_size", "tgs_select_tiles", "tgs_select_tiles_noalloc",
            "tgs_project_gaussians",
            "tgs_bin_tiles_workspace_size", "tgs_bin_tiles", "tgs_checkpoint_bytes", "tgs_set_forward_split", "tgs_render_sampled",
            "tgs_loss_sparse_ncc", "tgs_loss_sparse_ssim",
            "tgs_backward_sampled", "tgs_render_backward_sampled", "tgs_render_backward_sampled_stats", "tgs_error_stats_sampled", "tgs_project_backward", "tgs_project_backward_multi_workspace_size",
            "tgs_project_backward_multi", "tgs_project_backward_update",
            "tgs_render_batched_resident", "tgs_render_sampled_batched",
            "tgs_render_backward_batched", "tgs_render_backward_batched_stats", "tgs_hybrid_step_workspace_size", "tgs_hybrid_step",
            "tgs_mlp_param_count", "tgs_mlp_forward", "tgs_mlp_forward_tc", "tgs_mlp_tc_wait_drill", "tgs_mlp_backward_workspace_size",
            "tgs_mlp_backward", "tgs_mlp_backward_tc", "tgs_mlp_train_tc",
            "tgs_mlp_adam", "tgs_tile_observe", "tgs_tile_features", "tgs_tile_refresh",
            "tgs_view_error_sums", "tgs_sample_views", "tgs_accumulate_screen_grad",
            "tgs_density_control_workspace_size", "tgs_density_control"]


def _check(fn, status):
    if status != OK:
        raise TgsError(fn, status)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def version() -> str:
    return _lib.tgs_version().decode()


def graph_count_kernels(graph) -> int:
    """Kernel nodes in a captured torch.cuda.CUDAGraph."""
    return int(_lib.tgs_graph_count_kernels(C.c_void_p(graph.raw_cuda_graph())))


def advance_counters(iter_dev=None, step_dev=None, stream=None):
    _check("tgs_advance_counters", _lib.tgs_advance_counters(_ptr(iter_dev), _ptr(step_dev), _stream(stream)))


def device_check() -> None:
    _check("tgs_device_check", _lib.tgs_device_check())


def camera(cam: dict) -> Camera:
    c = Camera()
    vm = [float(v) for v in torch.as_tensor(cam["viewmat"], dtype=torch.float64).reshape(16).tolist()]
    c.viewmat = (C.c_float * 16)(*vm)
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.znear = float(cam.get("znear", 0.2))
    return c


def camera_array(cams, device="cuda") -> torch.Tensor:
    """Device array of tgs_camera structs (a uint8 tensor of len(cams) *
    sizeof(tgs_camera) bytes), for the calls that take one camera per view."""
    arr = (Camera * len(cams))(*[c if isinstance(c, Camera) else camera(c) for c in cams])
    return torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(device)


_GEO = ("means", "log_scales", "quats", "opacity_logits")
_GEO_WIDTH = {"means": 3, "log_scales": 3, "quats": 4, "opacity_logits": 1}


def _geo_ptrs(g: dict):
    """Device pointers of the four geometric fields and their geo_stride: 0
    when each is a contiguous array, else the common row stride (in floats)
    of four views into one array of rows (see ``geo_rows``)."""
    ts = [g[k] for k in _GEO]
    if all(t.is_contiguous() for t in ts):
        return [_ptr(t) for t in ts], 0
    n = ts[0].shape[0]
    rs = {t.stride(0) for t in ts}
    if len(rs) != 1:
        raise ValueError("geometric fields: one row stride for all four, or four contiguous arrays")
    stride = rs.pop()
    for k, t in zip(_GEO, ts):
        if not t.is_cuda or t.dtype != torch.float32 or t.shape[0] != n:
            raise ValueError(f"{k}: expected a float32 CUDA tensor of {n} rows")
        if _GEO_WIDTH[k] > 1 and (t.dim() != 2 or t.shape[1] != _GEO_WIDTH[k] or t.stride(1) != 1):
            raise ValueError(f"{k}: expected [{n}, {_GEO_WIDTH[k]}] with unit inner stride")
    return [t.data_ptr() for t in ts], int(stride)


def geo_rows(n: int, device="cuda", stride: int = 16, dtype=torch.float32) -> dict:
    """The geometric fields of n Gaussians as views into one [n, stride]
    array of rows (means at + 0, log_scales at + 3, opacity_logits at + 6,
    quats at + 8; zero-filled)."""
    if stride % 4 or stride < 12:
        raise ValueError("stride: a multiple of 4, at least 12")
    rows = torch.zeros(n, stride, dtype=dtype, device=device)
    return {"means": rows[:, 0:3], "log_scales": rows[:, 3:6], "opacity_logits": rows[:, 6],
            "quats": rows[:, 8:12]}


def gaussians(g: dict, sh_degree: int = 3) -> Gaussians:
    p, gs = _geo_ptrs(g)
    return Gaussians(p[0], p[1], p[2], p[3], _ptr(g["sh"]), int(g["means"].shape[0]), int(sh_degree), gs)


def param_ptrs(g: dict) -> ParamPtrs:
    p, gs = _geo_ptrs(g)
    return ParamPtrs(p[0], p[1], p[2], p[3], _ptr(g["sh"]), gs)


def projected(p: dict) -> Projected:
    return Projected(_ptr(p["xy"]), _ptr(p["conic_opac"]), _ptr(p["rgb"]), _ptr(p["depth"]), _ptr(p["radius"]))


# ----------------------------------------------------------------------------
# entry points
# ----------------------------------------------------------------------------

def select_tiles_workspace_size(width: int, height: int) -> int:
    return int(_lib.tgs_select_tiles_workspace_size(width, height))


def select_tiles(err_map, age_map, width, height, n_select, n_pix, sampling, seed, it, view, workspace,
                 active_tiles, n_active, tile_rank, pix_off, pix_idx, stream=None, iter_dev=None):
    cfg = Sampling(*sampling)
    _check("tgs_select_tiles", _lib.tgs_select_tiles(
        _ptr(err_map), _ptr(age_map), int(width), int(height), int(n_select), int(n_pix), C.byref(cfg),
        int(seed) & (2**64 - 1), int(it) & (2**64 - 1), _ptr(iter_dev), int(view), _ptr(workspace),
        workspace.numel(),
        _ptr(active_tiles), _ptr(n_active), _ptr(tile_rank), _ptr(pix_off), _ptr(pix_idx), _stream(stream)))


def select_tiles_noalloc(err_map, age_map, width, height, n_select, n_pix, sampling, seed, it, view, active_tiles,
                         n_active, tile_rank, pix_off, pix_idx, stream=None, iter_dev=None):
    """select_tiles with the library's built-in scratch instead of a workspace
    (for callers that cannot allocate device memory; see the C header)."""
    cfg = Sampling(*sampling)
    _check("tgs_select_tiles_noalloc", _lib.tgs_select_tiles_noalloc(
        _ptr(err_map), _ptr(age_map), int(width), int(height), int(n_select), int(n_pix), C.byref(cfg),
        int(seed) & (2**64 - 1), int(it) & (2**64 - 1), _ptr(iter_dev), int(view), _ptr(active_tiles),
        _ptr(n_active), _ptr(tile_rank), _ptr(pix_off), _ptr(pix_idx), _stream(stream)))


def project_gaussians(g: dict, cam, tile_rank, out: dict, sh_degree=3, stream=None):
    gs = gaussians(g, sh_degree)
    cc = cam if isinstance(cam, Camera) else camera(cam)
    pr = projected(out)
    _check("tgs_project_gaussians", _lib.tgs_project_gaussians(C.byref(gs), C.byref(cc), _ptr(tile_rank),
                                                               C.byref(pr), _stream(stream)))


def bin_tiles_workspace_size(n: int, capacity: int, n_active_max: int) -> int:
    return int(_lib.tgs_bin_tiles_workspace_size(int(n), int(capacity), int(n_active_max)))


def bin_tiles(proj: dict, n, cam, tile_rank, n_active_max, workspace, capacity, vals, keys, tile_ranges, n_isect,
              stream=None):
    pr = projected(proj)
    cc = cam if isinstance(cam, Camera) else camera(cam)
    _check("tgs_bin_tiles", _lib.tgs_bin_tiles(
        C.byref(pr), int(n), C.byref(cc), _ptr(tile_rank), int(n_active_max), _ptr(workspace), workspace.numel(),
        int(capacity), _ptr(vals), _ptr(keys), _ptr(tile_ranges), _ptr(n_isect), _stream(stream)))


def set_forward_split(groups: int) -> None:
    """Tuning knob of the checkpointed forward: 0 picks the split walk's
    group count per launch; 1 (sequential), 2 or 4 fix it process-wide."""
    _check("tgs_set_forward_split", _lib.tgs_set_forward_split(int(groups)))


def checkpoint_bytes(n_active_max: int, n_pix_max: int, n_slots: int) -> int:
    return int(_lib.tgs_checkpoint_bytes(int(n_active_max), int(n_pix_max), int(n_slots)))


def checkpoints(data, n_slots: int, stride: int, rgb, tile_last=None) -> Checkpoints:
    """data: float32 device tensor of checkpoint_bytes(...) / 4 elements; rgb:
    the forward's rgb output tensor; tile_last: optional int32 [n_active_max]."""
    return Checkpoints(_ptr(data), int(n_slots), int(stride), _ptr(rgb), _ptr(tile_last))


def _ck(ckpt):
    return C.byref(ckpt) if ckpt is not None else None


def render_sampled(proj: dict, tile_ranges, vals, active_tiles, n_active, n_active_max, pix_off, pix_idx,
                   n_pix_max, cam, bg, rgb, T_final, n_last, stream=None, ckpt=None):
    pr = projected(proj)
    cc = cam if isinstance(cam, Camera) else camera(cam)
    bgv = (C.c_float * 3)(*[float(b) for b in bg])
    _check("tgs_render_sampled", _lib.tgs_render_sampled(
        C.byref(pr), _ptr(tile_ranges), _ptr(vals), _ptr(active_tiles), _ptr(n_active), int(n_active_max),
        _ptr(pix_off), _ptr(pix_idx), int(n_pix_max), C.byref(cc), bgv, _ptr(rgb), _ptr(T_final), _ptr(n_last),
        _ck(ckpt), _stream(stream)))


def loss_sparse_ncc(rgb, target, width, height, active_tiles, n_active, n_active_max, pix_off, pix_idx, n_pix_max,
                    loss_params, err_map, age_map, dL_drgb, lambda_tile, err_pix, loss, stream=None, structure="ncc"):
    """The fused sparse loss; structure="ssim" takes the S-SSIM variant
    (tgs_loss_sparse_ssim) in place of the sparse NCC term."""
    vals = [float(v) for v in loss_params]
    if len(vals) == 3:
        vals.append(1.0)  # one view
    lp = LossParams(*vals)
    name = {"ncc": "tgs_loss_sparse_ncc", "ssim": "tgs_loss_sparse_ssim"}[structure]
    _check(name, getattr(_lib, name)(
        _ptr(rgb), _ptr(target), int(width), int(height), _ptr(active_tiles), _ptr(n_active), int(n_active_max),
        _ptr(pix_off), _ptr(pix_idx), int(n_pix_max), C.byref(lp), _ptr(err_map), _ptr(age_map), _ptr(dL_drgb),
        _ptr(lambda_tile), _ptr(err_pix), _ptr(loss), _stream(stream)))


def loss_sparse_ssim(rgb, target, width, height, active_tiles, n_active, n_active_max, pix_off, pix_idx, n_pix_max,
                     loss_params, err_map, age_map, dL_drgb, lambda_tile, err_pix, loss, stream=None):
    """The fused sparse loss with Table 4's S-SSIM structure term."""
    loss_sparse_ncc(rgb, target, width, height, active_tiles, n_active, n_active_max, pix_off, pix_idx, n_pix_max,
                    loss_params, err_map, age_map, dL_drgb, lambda_tile, err_pix, loss, stream=stream,
                    structure="ssim")


def backward_sampled(g: dict, cam, proj: dict, tile_ranges, vals, active_tiles, n_active, n_active_max, pix_off,
                     pix_idx, n_pix_max, bg, T_final, n_last, dL_drgb, grad2d, grads: dict, touched,
                     write_untouched=True, sh_degree=3, stream=None, ckpt=None):
    gs = gaussians(g, sh_degree)
    cc = cam if isinstance(cam, Camera) else camera(cam)
    pr = projected(proj)
    gp = param_ptrs(grads)
    bgv = (C.c_float * 3)(*[float(b) for b in bg])
    _check("tgs_backward_sampled", _lib.tgs_backward_sampled(
        C.byref(gs), C.byref(cc), C.byref(pr), _ptr(tile_ranges), _ptr(vals), _ptr(active_tiles), _ptr(n_active),
        int(n_active_max), _ptr(pix_off), _ptr(pix_idx), int(n_pix_max), bgv, _ptr(T_final), _ptr(n_last),
        _ptr(dL_drgb), _ptr(grad2d), C.byref(gp), _ptr(touched), 1 if write_untouched else 0, _ck(ckpt),
        _stream(stream)))


def render_backward_sampled_stats(proj: dict, tile_ranges, vals, active_tiles, n_active, n_active_max, pix_off,
                                  pix_idx, n_pix_max, cam, bg, T_final, n_last, dL_drgb, grad2d, err_pix, stats,
                                  accumulate=False, stream=None, ckpt=None):
    """render_backward_sampled plus Eq. 12's statistics of the same pixels
    into stats [N,4] (zeroed first unless accumulate)."""
    pr = projected(proj)
    cc = cam if isinstance(cam, Camera) else camera(cam)
    bgv = (C.c_float * 3)(*[float(b) for b in bg])
    _check("tgs_render_backward_sampled_stats", _lib.tgs_render_backward_sampled_stats(
        C.byref(pr), _ptr(tile_ranges), _ptr(vals), _ptr(active_tiles), _ptr(n_active), int(n_active_max),
        _ptr(pix_off), _ptr(pix_idx), int(n_pix_max), C.byref(cc), bgv, _ptr(T_final), _ptr(n_last), _ptr(dL_drgb),
        _ptr(grad2d), int(grad2d.shape[0]), _ck(ckpt), _ptr(err_pix), _ptr(stats), 1 if accumulate else 0,
        _stream(stream)))


def render_backward_sampled(proj: dict, tile_ranges, vals, active_tiles, n_active, n_active_max, pix_off, pix_idx,
                            n_pix_max, cam, bg, T_final, n_last, dL_drgb, grad2d, stream=None, ckpt=None):
    pr = projected(proj)
    cc = cam if isinstance(cam, Camera) else camera(cam)
    bgv = (C.c_float * 3)(*[float(b) for b in bg])
    _check("tgs_render_backward_sampled", _lib.tgs_render_backward_sampled(
        C.byref(pr), _ptr(tile_ranges), _ptr(vals), _ptr(active_tiles), _ptr(n_active), int(n_active_max),
        _ptr(pix_off), _ptr(pix_idx), int(n_pix_max), C.byref(cc), bgv, _ptr(T_final), _ptr(n_last), _ptr(dL_drgb),
        _ptr(grad2d), int(grad2d.shape[0]), _ck(ckpt), _stream(stream)))


def error_stats_sampled(proj: dict, tile_ranges, vals, active_tiles, n_active, n_active_max, pix_off, pix_idx,
                        n_pix_max, cam, n_last, err_pix, stats, accumulate=False, stream=None):
    """stats [N, 4] float: (sum e w, sum w, sum D w, 0) per Gaussian (Sec. 3.8)."""
    pr = projected(proj)
    cc = cam if isinstance(cam, Camera) else camera(cam)
    _check("tgs_error_stats_sampled", _lib.tgs_error_stats_sampled(
        C.byref(pr), _ptr(tile_ranges), _ptr(vals), _ptr(active_tiles), _ptr(n_active), int(n_active_max),
        _ptr(pix_off), _ptr(pix_idx), int(n_pix_max), C.byref(cc), _ptr(n_last), _ptr(err_pix), _ptr(stats),
        int(stats.shape[0]), 1 if accumulate else 0, _stream(stream)))


def project_backward(g: dict, cam, proj: dict, grad2d, grads: dict, touched, write_untouched=True,
                     accumulate=False, view_row=None, sh_degree=3, stream=None):
    gs = gaussians(g, sh_degree)
    cc = cam if isinstance(cam, Camera) else camera(cam)
    pr = projected(proj)
    gp = param_ptrs(grads)
    _check("tgs_project_backward", _lib.tgs_project_backward(
        C.byref(gs), C.byref(cc), C.byref(pr), _ptr(grad2d), C.byref(gp), _ptr(touched),
        1 if write_untouched else 0, 1 if accumulate else 0, _ptr(view_row), _stream(stream)))


class MultiAdjoint:
    """Marshalled arguments of project_backward_multi (the host pointer arrays
    are built once; the device buffers they point to must stay alive)."""

    def __init__(self, cams: list, radius: list, grad2d: list, view_rows: list | None = None):
        K = len(cams)
        self.K = K
        self.cams = (Camera * K)(*[c if isinstance(c, Camera) else camera(c) for c in cams])
        self.radius = (C.c_void_p * K)(*[_ptr(r) for r in radius])
        self.grad2d = (C.c_void_p * K)(*[_ptr(g) for g in grad2d])
        self.rows = None if view_rows is None else (C.c_void_p * K)(*[_ptr(r) for r in view_rows])


def project_backward_multi_workspace_size(n: int) -> int:
    return int(_lib.tgs_project_backward_multi_workspace_size(int(n)))


def project_backward_multi(g: dict, adj: MultiAdjoint, grads: dict, touched, write_untouched=False, sh_degree=3,
                           workspace=None, stream=None):
    gs = gaussians(g, sh_degree)
    gp = param_ptrs(grads)
    if workspace is None:
        workspace = torch.empty(project_backward_multi_workspace_size(gs.n), dtype=torch.uint8,
                                device=g["means"].device)
    _check("tgs_project_backward_multi", _lib.tgs_project_backward_multi(
        C.byref(gs), adj.K, adj.cams, adj.radius, adj.grad2d, C.byref(gp), _ptr(touched),
        1 if write_untouched else 0, adj.rows, _ptr(workspace), workspace.numel(), _stream(stream)))


def view_batch(views: list) -> C.Array:
    """views: dicts with the per-view fields of tgs_view_batch (proj, tile_ranges,
    vals, active_tiles, n_active, n_active_max, pix_off, pix_idx, n_pix_max, cam,
    bg, rgb, T_final, n_last, optionally ckpt (a Checkpoints) and, for the
    backward, dL_drgb, grad2d)."""
    arr = (ViewBatch * len(views))()
    for k, w in enumerate(views):
        b = arr[k]
        b.proj = projected(w["proj"])
        b.tile_ranges, b.vals = _ptr(w["tile_ranges"]), _ptr(w["vals"])
        b.active_tiles, b.n_active = _ptr(w["active_tiles"]), _ptr(w["n_active"])
        b.n_active_max = int(w["n_active_max"])
        b.pix_off, b.pix_idx, b.n_pix_max = _ptr(w["pix_off"]), _ptr(w["pix_idx"]), int(w["n_pix_max"])
        b.cam = w["cam"] if isinstance(w["cam"], Camera) else camera(w["cam"])
        b.bg = (C.c_float * 3)(*[float(x) for x in w.get("bg", (0.0, 0.0, 0.0))])
        b.rgb, b.T_final, b.n_last = _ptr(w["rgb"]), _ptr(w["T_final"]), _ptr(w["n_last"])
        b.dL_drgb, b.grad2d = _ptr(w.get("dL_drgb")), _ptr(w.get("grad2d"))
        b.n_gaussians = int(w["grad2d"].shape[0]) if w.get("grad2d") is not None else 0
        if w.get("ckpt") is not None:
            b.ckpt = w["ckpt"]
    return arr


def render_batched_resident(n_pix_max: int, backward) -> int:
    """backward: 0 / False the forward, 1 / True the whole-tile backward, 2 the
    backward in pieces (with checkpoints)."""
    out = _i32(0)
    _check("tgs_render_batched_resident", _lib.tgs_render_batched_resident(int(n_pix_max), int(backward),
                                                                             C.byref(out)))
    return int(out.value)


def render_sampled_batched(views, grid_ctas, counter, stream=None):
    arr = views if isinstance(views, C.Array) else view_batch(views)
    _check("tgs_render_sampled_batched", _lib.tgs_render_sampled_batched(arr, len(arr), int(grid_ctas),
                                                                           _ptr(counter), _stream(stream)))


def render_backward_batched_stats(views, grid_ctas, counter, err_pix: list, stats, accumulate=False, stream=None):
    """The batched backward with Eq. 12's statistics of every view's sampled
    pixels into stats [N,4] (zeroed first unless accumulate)."""
    arr = views if isinstance(views, C.Array) else view_batch(views)
    errs = (_p * len(arr))(*[_ptr(e) for e in err_pix])
    _check("tgs_render_backward_batched_stats", _lib.tgs_render_backward_batched_stats(
        arr, len(arr), int(grid_ctas), _ptr(counter), errs, _ptr(stats), int(stats.shape[0]), 1 if accumulate else 0,
        _stream(stream)))


def render_backward_batched(views, grid_ctas, counter, stream=None):
    arr = views if isinstance(views, C.Array) else view_batch(views)
    _check("tgs_render_backward_batched", _lib.tgs_render_backward_batched(arr, len(arr), int(grid_ctas),
                                                                             _ptr(counter), _stream(stream)))


def hybrid_step_workspace_size(n: int) -> int:
    return int(_lib.tgs_hybrid_step_workspace_size(int(n)))


def opt_struct(opt: dict) -> Opt:
    o = Opt()
    o.lr = (C.c_float * 6)(*[float(x) for x in opt["lr"]])
    o.beta1, o.beta2 = float(opt["beta1"]), float(opt["beta2"])
    o.eps_adam, o.eps_lm = float(opt["eps_adam"]), float(opt["eps_lm"])
    o.mode = int(opt["mode"])
    return o


def project_backward_update(params: dict, adj, m: dict, v: dict, touched, opt: dict, step=1, step_dev=None,
                            sh_degree=3, workspace=None, stream=None):
    P, M, V = param_ptrs(params), param_ptrs(m), param_ptrs(v)
    n = int(params["means"].shape[0])
    if workspace is None:
        workspace = torch.empty(project_backward_multi_workspace_size(n), dtype=torch.uint8,
                                device=params["means"].device)
    o = opt_struct(opt)
    _check("tgs_project_backward_update", _lib.tgs_project_backward_update(
        C.byref(P), n, int(sh_degree), adj.K, adj.cams, adj.radius, adj.grad2d, C.byref(M), C.byref(V),
        _ptr(touched), C.byref(o), int(step), _ptr(step_dev), _ptr(workspace), workspace.numel(),
        _stream(stream)))


def hybrid_step(params: dict, grads: dict, m: dict, v: dict, n, touched, view_rows, k_rows, step, opt,
                workspace=None, stream=None, step_dev=None):
    P, G, M, V = param_ptrs(params), param_ptrs(grads), param_ptrs(m), param_ptrs(v)
    if workspace is None:
        workspace = torch.empty(hybrid_step_workspace_size(n), dtype=torch.uint8, device=params["means"].device)
    o = opt_struct(opt)
    _check("tgs_hybrid_step", _lib.tgs_hybrid_step(
        C.byref(P), C.byref(G), C.byref(M), C.byref(V), int(n), _ptr(touched), _ptr(view_rows), int(k_rows),
        int(step), _ptr(step_dev), C.byref(o), _ptr(workspace), workspace.numel(), _stream(stream)))


# ----------------------------------------------------------------------------
# tile-error predictor
# ----------------------------------------------------------------------------

def mlp_param_count() -> int:
    return int(_lib.tgs_mlp_param_count())


def mlp_struct(net: dict) -> Mlp:
    """net: w1, w2, w3 (int16 tensors holding bf16 bits), b1, b2, b3 (float32)."""
    return Mlp(_ptr(net["w1"]), _ptr(net["b1"]), _ptr(net["w2"]), _ptr(net["b2"]), _ptr(net["w3"]), _ptr(net["b3"]))


def mlp_forward(net: dict, x, y, h1=None, h2=None, stream=None):
    m = mlp_struct(net)
    _check("tgs_mlp_forward", _lib.tgs_mlp_forward(C.byref(m), int(x.shape[0]), _ptr(x), _ptr(y), _ptr(h1), _ptr(h2),
                                                   _stream(stream)))


def mlp_forward_tc(net: dict, x, y, h1=None, h2=None, status=None, stream=None):
    m = mlp_struct(net)
    _check("tgs_mlp_forward_tc", _lib.tgs_mlp_forward_tc(C.byref(m), int(x.shape[0]), _ptr(x), _ptr(y), _ptr(h1),
                                                         _ptr(h2), _ptr(status), _stream(stream)))


def mlp_tc_wait_drill(status, stream=None):
    _check("tgs_mlp_tc_wait_drill", _lib.tgs_mlp_tc_wait_drill(_ptr(status), _stream(stream)))


def mlp_backward_workspace_size(rows: int) -> int:
    return int(_lib.tgs_mlp_backward_workspace_size(int(rows)))


def mlp_backward(net: dict, x, h1, h2, y, target, grads, loss, workspace=None, stream=None, rows_dev=None):
    m = mlp_struct(net)
    if workspace is None:
        workspace = torch.empty(mlp_backward_workspace_size(x.shape[0]), dtype=torch.uint8, device=x.device)
    _check("tgs_mlp_backward", _lib.tgs_mlp_backward(C.byref(m), int(x.shape[0]), _ptr(rows_dev), _ptr(x), _ptr(h1),
                                                     _ptr(h2), _ptr(y), _ptr(target), _ptr(grads), _ptr(loss),
                                                     _ptr(workspace), workspace.numel(), _stream(stream)))


def mlp_backward_tc(net: dict, x, h1, h2, y, target, grads, loss, status=None, workspace=None, stream=None,
                    rows_dev=None):
    """mlp_backward with the weight gradients on the tcgen05 tensor cores."""
    m = mlp_struct(net)
    if workspace is None:
        workspace = torch.empty(mlp_backward_workspace_size(x.shape[0]), dtype=torch.uint8, device=x.device)
    _check("tgs_mlp_backward_tc", _lib.tgs_mlp_backward_tc(
        C.byref(m), int(x.shape[0]), _ptr(rows_dev), _ptr(x), _ptr(h1), _ptr(h2), _ptr(y), _ptr(target), _ptr(grads),
        _ptr(loss), _ptr(status), _ptr(workspace), workspace.numel(), _stream(stream)))


def mlp_train_tc(net: dict, x, target, grads, loss, y=None, status=None, stream=None, rows_dev=None):
    """The loss's gradient with the forward recomputed in the same tcgen05
    kernel (no stored activations); y (optional) receives the outputs."""
    m = mlp_struct(net)
    _check("tgs_mlp_train_tc", _lib.tgs_mlp_train_tc(
        C.byref(m), int(x.shape[0]), _ptr(rows_dev), _ptr(x), _ptr(target), _ptr(y), _ptr(grads), _ptr(loss),
        _ptr(status), _stream(stream)))


def mlp_adam(params, grads, m, v, step, lr, beta1, beta2, eps, net: dict, stream=None):
    _check("tgs_mlp_adam", _lib.tgs_mlp_adam(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(step), float(lr),
                                             float(beta1), float(beta2), float(eps), _ptr(net["w1"]),
                                             _ptr(net["w2"]), _ptr(net["w3"]), _stream(stream)))


# ----------------------------------------------------------------------------
# tile memory and features of the tile-error predictor
# ----------------------------------------------------------------------------

def tile_observe(active_tiles, n_active, n_active_max, pix_off, tile_ranges, T_final, err_pix, mem, mem_iter,
                 target=None, it=0, iter_dev=None, residual=False, stream=None):
    _check("tgs_tile_observe", _lib.tgs_tile_observe(
        _ptr(active_tiles), _ptr(n_active), int(n_active_max), _ptr(pix_off), _ptr(tile_ranges), _ptr(T_final),
        _ptr(err_pix), int(it) & (2**64 - 1), _ptr(iter_dev), _ptr(mem), _ptr(mem_iter), _ptr(target),
        1 if residual else 0, _stream(stream)))


def tile_features(mem, mem_iter, cam, x, rows=None, n_rows=None, n_rows_max=None, view_cos=1.0, it=0,
                  iter_dev=None, stream=None):
    cc = cam if isinstance(cam, Camera) else camera(cam)
    nmax = int(n_rows_max if n_rows_max is not None else x.shape[0])
    _check("tgs_tile_features", _lib.tgs_tile_features(
        _ptr(mem), _ptr(mem_iter), _ptr(rows), _ptr(n_rows), nmax, C.byref(cc), float(view_cos),
        int(it) & (2**64 - 1), _ptr(iter_dev), _ptr(x), _stream(stream)))


def tile_refresh(pred, err_map, width, height, base=None, stream=None):
    _check("tgs_tile_refresh", _lib.tgs_tile_refresh(_ptr(pred), _ptr(base), _ptr(err_map), int(width), int(height),
                                                     _stream(stream)))


def view_error_sums(err_maps, sums, stream=None):
    """err_maps [V,H,W] int16 (fp16 bit patterns, contiguous); sums [V] int64
    receives the exact totals of E * 2^24 (Eq. 5 times W H 2^24)."""
    V, H, W = (int(x) for x in err_maps.shape)
    if sums.dtype != torch.int64 or sums.numel() < V:
        raise ValueError("sums: int64 [V]")
    _check("tgs_view_error_sums", _lib.tgs_view_error_sums(_ptr(err_maps), V, H * W, W, H, _ptr(sums),
                                                           _stream(stream)))


def sample_views(err_sums, cams, k, lambda_d, lambda_theta, seed, it, stack, views, stream=None):
    """Geometry-aware draw of k views (Eqs. 5-6): err_sums [V] int64 from
    view_error_sums, cams from camera_array, stack [V] uint8 (in/out), views
    [k] int32 (anchor first, then the draws ascending)."""
    V = int(err_sums.numel())
    if stack.dtype != torch.uint8 or stack.numel() != V or views.dtype != torch.int32 or views.numel() < k:
        raise ValueError("stack: uint8 [V]; views: int32 [k]")
    if cams.dtype != torch.uint8 or cams.numel() != V * C.sizeof(Camera):
        raise ValueError("cams: camera_array of V cameras")
    _check("tgs_sample_views", _lib.tgs_sample_views(
        _ptr(err_sums), _ptr(cams), V, int(k), float(lambda_d), float(lambda_theta), int(seed) & (2**64 - 1),
        int(it) & (2**64 - 1), _ptr(stack), _ptr(views), _stream(stream)))


# ----------------------------------------------------------------------------
# error-driven density control (Sec. 3.8)
# ----------------------------------------------------------------------------

def accumulate_screen_grad(grad2d, accum, stream=None):
    """accum [N,2] += (|(dL/dx, dL/dy)|, 1) where the view's grad2d row is not zero."""
    _check("tgs_accumulate_screen_grad", _lib.tgs_accumulate_screen_grad(_ptr(grad2d), int(grad2d.shape[0]),
                                                                          _ptr(accum), _stream(stream)))


def density_control_workspace_size(n: int) -> int:
    return int(_lib.tgs_density_control_workspace_size(int(n)))


def density_params(lambda_eff, tau_grad, log_scale_split, opacity_logit_prune, topk_permille=800, final=False,
                   final_permille=900, eps=1e-8) -> DensityParams:
    return DensityParams(float(lambda_eff), float(eps), float(tau_grad), float(log_scale_split),
                         float(opacity_logit_prune), int(topk_permille), 1 if final else 0, int(final_permille))


def density_control(params: dict, m: dict, v: dict, stats, accum, cfg: DensityParams, params_out: dict, m_out: dict,
                    v_out: dict, capacity: int, n_out, src_out=None, workspace=None, sh_degree=3, stream=None):
    """One density-control step; n_out (device int64 [1]) receives the output
    count (rows past capacity are not written)."""
    n = int(params["means"].shape[0])
    if workspace is None:
        workspace = torch.empty(density_control_workspace_size(n), dtype=torch.uint8, device=params["means"].device)
    gs = gaussians(params, sh_degree)
    _check("tgs_density_control", _lib.tgs_density_control(
        C.byref(gs), C.byref(param_ptrs(m)), C.byref(param_ptrs(v)), _ptr(stats), _ptr(accum), C.byref(cfg),
        C.byref(param_ptrs(params_out)), C.byref(param_ptrs(m_out)), C.byref(param_ptrs(v_out)), int(capacity),
        _ptr(n_out), _ptr(src_out), _ptr(workspace), workspace.numel(), _stream(stream)))

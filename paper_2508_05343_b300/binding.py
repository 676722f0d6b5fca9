"""ctypes binding of libgabsplat.so: the C ABI declared in include/gabsplat.h, same names.

This module only marshals arguments (torch tensors -> device pointers, camera dicts -> structs,
the current CUDA stream).  Every step of the rasterizer runs in the library's CUDA kernels; there
is no fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgabsplat.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, GS_ERR_CUDA, GS_ERR_NONFINITE, GS_ERR_WORKSPACE = range(7)
GS_F32, GS_BF16 = 0, 1
GS_LOSS_L1, GS_LOSS_L2 = 0, 1
GS_FLAG_Z_ATTENUATION = 1
GS_TILE, GS_MAX_K, GS_MAX_SH_DEGREE, GS_MAX_VIEWS = 16, 8, 3, 16


class gs_prims(C.Structure):
    _fields_ = [("n", C.c_int), ("K", C.c_int), ("sh_degree", C.c_int), ("storage", C.c_int),
                ("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p), ("freqs", C.c_void_p), ("weights", C.c_void_p)]


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int), ("height", C.c_int),
                ("znear", C.c_float), ("zfar", C.c_float)]


class gs_config(C.Structure):
    _fields_ = [("eps2d", C.c_float), ("alpha_max", C.c_float), ("alpha_min", C.c_float), ("T_min", C.c_float),
                ("bg", C.c_float * 3), ("flags", C.c_uint)]


class gs_frame(C.Structure):
    _fields_ = [("n", C.c_int), ("K", C.c_int), ("sh_degree", C.c_int), ("width", C.c_int), ("height", C.c_int),
                ("storage", C.c_int), ("pair_capacity", C.c_ulonglong), ("ws", C.c_void_p), ("ws_bytes", C.c_size_t)]


class gs_prim_grads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("means", "scales", "quats", "opacity", "sh", "freqs", "weights", "means2d")]


class gs_densify_config(C.Structure):
    _fields_ = [(k, C.c_float) for k in ("grad_threshold", "dense_scale", "min_opacity", "max_scale", "split_divisor",
                                          "child_freq", "child_weight")]


class gs_prim_arrays(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("means", "scales", "quats", "opacity", "sh", "freqs", "weights")]


class gs_ws_views(C.Structure):
    _fields_ = [("records", C.c_void_p), ("touched", C.c_void_p), ("offsets", C.c_void_p),
                ("order", C.c_void_p), ("n_active", C.c_uint), ("keys_sorted", C.c_void_p),
                ("keys_unsorted", C.c_void_p), ("ranges", C.c_void_p), ("T_final", C.c_void_p),
                ("n_contrib", C.c_void_p), ("n_eval", C.c_void_p), ("n_reach", C.c_void_p), ("n_comp", C.c_void_p), ("grad2d", C.c_void_p), ("record_floats", C.c_int),
                ("grad2d_floats", C.c_int), ("tiles_x", C.c_int), ("tiles_y", C.c_int)]


class gs_view(C.Structure):
    _fields_ = [("prims", gs_prims), ("cam", gs_camera), ("out_rgb", C.c_void_p), ("out_T", C.c_void_p)]


class gs_batch_frame(C.Structure):
    _fields_ = [("max_views", C.c_int), ("K", C.c_int), ("sh_degree", C.c_int), ("storage", C.c_int),
                ("max_prims", C.c_ulonglong), ("max_tiles", C.c_ulonglong), ("max_pixels", C.c_ulonglong),
                ("pair_capacity", C.c_ulonglong), ("ws", C.c_void_p), ("ws_bytes", C.c_size_t)]


P_ = C.POINTER
SIGNATURES = {
    "gabsplat_workspace_size": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong]),
    "gabsplat_workspace_init": (C.c_int, [P_(gs_frame), C.c_void_p]),
    "gabsplat_preprocess": (C.c_int, [P_(gs_frame), P_(gs_prims), P_(gs_camera), P_(gs_config), C.c_void_p]),
    "gabsplat_bin_sort": (C.c_int, [P_(gs_frame), C.c_void_p]),
    "gabsplat_render_fwd": (C.c_int, [P_(gs_frame), C.c_void_p, C.c_void_p, C.c_void_p]),
    "gabsplat_render_freq_map": (C.c_int, [P_(gs_frame), C.c_void_p, C.c_void_p]),
    "gabsplat_render_fwd_only": (C.c_int, [P_(gs_frame), C.c_void_p, C.c_void_p, C.c_void_p]),
    "gabsplat_render_fwd_stats": (C.c_int, [P_(gs_frame), C.c_void_p, C.c_void_p, C.c_void_p]),
    "gabsplat_densify_accumulate": (C.c_int, [P_(gs_frame), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gabsplat_densify_scratch_bytes": (C.c_size_t, [C.c_int]),
    "gabsplat_densify": (C.c_int, [P_(gs_prims), C.c_void_p, C.c_void_p, C.c_void_p, P_(gs_densify_config),
                                   P_(gs_prim_arrays), C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gabsplat_reset_opacity_weights": (C.c_int, [P_(gs_prim_arrays), C.c_int, C.c_int, C.c_int, C.c_float, C.c_float,
                                                 C.c_void_p]),
    "gabsplat_render_bwd": (C.c_int, [P_(gs_frame), C.c_void_p, P_(gs_prim_grads), C.c_void_p]),
    "gabsplat_render_bwd_2d": (C.c_int, [P_(gs_frame), C.c_void_p, C.c_void_p]),
    "gabsplat_preprocess_bwd": (C.c_int, [P_(gs_frame), P_(gs_prim_grads), C.c_void_p]),
    "gabsplat_render_bwd_2d_zero": (C.c_int, [P_(gs_frame), C.c_void_p, P_(gs_prim_grads), C.c_void_p]),
    "gabsplat_preprocess_bwd_prezeroed": (C.c_int, [P_(gs_frame), P_(gs_prim_grads), C.c_void_p]),
    "gabsplat_loss_scratch_bytes": (C.c_size_t, [C.c_longlong]),
    "gabsplat_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "gabsplat_loss_l1_dssim_scratch_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int]),
    "gabsplat_loss_l1_dssim": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_float, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]),
    "gabsplat_loss_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_void_p]),
    "gabsplat_device_status": (C.c_int, [P_(gs_frame), P_(C.c_int), P_(C.c_ulonglong), C.c_void_p]),
    "gabsplat_workspace_views": (C.c_int, [P_(gs_frame), P_(gs_ws_views)]),
    "gabsplat_batch_workspace_size": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_ulonglong, C.c_ulonglong,
                                                   C.c_ulonglong, C.c_ulonglong]),
    "gabsplat_batch_workspace_init": (C.c_int, [P_(gs_batch_frame), C.c_void_p]),
    "gabsplat_render_batch": (C.c_int, [P_(gs_batch_frame), P_(gs_view), C.c_int, P_(gs_config), C.c_void_p]),
    "gabsplat_batch_status_copy": (C.c_int, [P_(gs_batch_frame), C.c_void_p, C.c_void_p]),
    "gabsplat_batch_graph_create": (C.c_int, [P_(gs_batch_frame), P_(gs_config), C.c_void_p, P_(C.c_void_p)]),
    "gabsplat_batch_graph_launch": (C.c_int, [C.c_void_p, P_(gs_view), C.c_int, C.c_void_p]),
    "gabsplat_batch_graph_destroy": (None, [C.c_void_p]),
    "gabsplat_status_string": (C.c_char_p, [C.c_int]),
    "gabsplat_version": (C.c_char_p, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2508_05343_b300.build`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class GabsplatError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__(f"{fn}: {status_string(status)} ({status})")
        self.status = status


def _check(fn, st):
    if st != GS_OK:
        raise GabsplatError(fn, st)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


# ---- the ABI, same names --------------------------------------------------------------------
def gabsplat_workspace_size(n, K, sh_degree, width, height, pair_capacity):
    return int(lib.gabsplat_workspace_size(n, K, sh_degree, width, height, pair_capacity))


def gabsplat_workspace_init(frame, stream=None):
    _check("gabsplat_workspace_init", lib.gabsplat_workspace_init(C.byref(frame), _stream(stream)))


def gabsplat_preprocess(frame, prims, cam, cfg, stream=None):
    _check("gabsplat_preprocess", lib.gabsplat_preprocess(C.byref(frame), C.byref(prims), C.byref(cam),
                                                          C.byref(cfg), _stream(stream)))


def gabsplat_bin_sort(frame, stream=None):
    _check("gabsplat_bin_sort", lib.gabsplat_bin_sort(C.byref(frame), _stream(stream)))


def gabsplat_render_fwd(frame, out_rgb, out_T=None, stream=None):
    _check("gabsplat_render_fwd", lib.gabsplat_render_fwd(C.byref(frame), _ptr(out_rgb), _ptr(out_T), _stream(stream)))


def gabsplat_render_fwd_stats(frame, out_rgb, out_T=None, stream=None):
    _check("gabsplat_render_fwd_stats", lib.gabsplat_render_fwd_stats(C.byref(frame), _ptr(out_rgb), _ptr(out_T),
                                                                       _stream(stream)))


def gabsplat_render_fwd_only(frame, out_rgb, out_T=None, stream=None):
    _check("gabsplat_render_fwd_only", lib.gabsplat_render_fwd_only(C.byref(frame), _ptr(out_rgb), _ptr(out_T),
                                                                    _stream(stream)))


def gabsplat_render_freq_map(frame, out_map, stream=None):
    _check("gabsplat_render_freq_map", lib.gabsplat_render_freq_map(C.byref(frame), _ptr(out_map), _stream(stream)))


def gabsplat_render_bwd(frame, dL_drgb, grads, stream=None):
    _check("gabsplat_render_bwd", lib.gabsplat_render_bwd(C.byref(frame), _ptr(dL_drgb), C.byref(grads),
                                                          _stream(stream)))


def gabsplat_render_bwd_2d(frame, dL_drgb, stream=None):
    _check("gabsplat_render_bwd_2d", lib.gabsplat_render_bwd_2d(C.byref(frame), _ptr(dL_drgb), _stream(stream)))


def gabsplat_preprocess_bwd(frame, grads, stream=None):
    _check("gabsplat_preprocess_bwd", lib.gabsplat_preprocess_bwd(C.byref(frame), C.byref(grads), _stream(stream)))


def gabsplat_render_bwd_2d_zero(frame, dL_drgb, grads, stream=None):
    _check("gabsplat_render_bwd_2d_zero", lib.gabsplat_render_bwd_2d_zero(C.byref(frame), _ptr(dL_drgb),
                                                                          C.byref(grads), _stream(stream)))


def gabsplat_preprocess_bwd_prezeroed(frame, grads, stream=None):
    _check("gabsplat_preprocess_bwd_prezeroed",
           lib.gabsplat_preprocess_bwd_prezeroed(C.byref(frame), C.byref(grads), _stream(stream)))


def gabsplat_loss_scratch_bytes(count):
    return int(lib.gabsplat_loss_scratch_bytes(count))


def gabsplat_loss(image, target, kind, loss_out, dL_dimage, scratch, stream=None):
    _check("gabsplat_loss", lib.gabsplat_loss(_ptr(image), _ptr(target), image.numel(), kind, _ptr(loss_out),
                                              _ptr(dL_dimage), _ptr(scratch), _stream(stream)))


def gabsplat_loss_l1_dssim_scratch_bytes(channels, height, width):
    return int(lib.gabsplat_loss_l1_dssim_scratch_bytes(channels, height, width))


def gabsplat_loss_l1_dssim(image, target, lam, loss_out, dL_dimage, scratch, stream=None):
    """image, target: [C][H][W] float32 device tensors; lam: the D-SSIM weight (0.2 in the paper)."""
    Cc, H, W = image.shape
    _check("gabsplat_loss_l1_dssim", lib.gabsplat_loss_l1_dssim(_ptr(image), _ptr(target), Cc, H, W, lam,
                                                                _ptr(loss_out), _ptr(dL_dimage), _ptr(scratch),
                                                                _stream(stream)))


def gabsplat_loss_noalloc(image, target, kind, loss_out, dL_dimage, stream=None):
    _check("gabsplat_loss_noalloc", lib.gabsplat_loss_noalloc(_ptr(image), _ptr(target), image.numel(), kind,
                                                              _ptr(loss_out), _ptr(dL_dimage), _stream(stream)))


def gabsplat_device_status(frame, stream=None):
    st, pairs = C.c_int(0), C.c_ulonglong(0)
    _check("gabsplat_device_status", lib.gabsplat_device_status(C.byref(frame), C.byref(st), C.byref(pairs),
                                                                _stream(stream)))
    return int(st.value), int(pairs.value)


def gabsplat_workspace_views(frame):
    v = gs_ws_views()
    _check("gabsplat_workspace_views", lib.gabsplat_workspace_views(C.byref(frame), C.byref(v)))
    return v


def gabsplat_batch_workspace_size(max_views, K, sh_degree, max_prims, max_tiles, max_pixels, pair_capacity):
    return int(lib.gabsplat_batch_workspace_size(max_views, K, sh_degree, max_prims, max_tiles, max_pixels,
                                                 pair_capacity))


def gabsplat_batch_workspace_init(frame, stream=None):
    _check("gabsplat_batch_workspace_init", lib.gabsplat_batch_workspace_init(C.byref(frame), _stream(stream)))


def _view_array(views):
    arr = (gs_view * max(1, len(views)))()
    for i, v in enumerate(views):
        arr[i] = v
    return arr


def gabsplat_render_batch(frame, views, cfg, stream=None):
    _check("gabsplat_render_batch", lib.gabsplat_render_batch(C.byref(frame), _view_array(views), len(views),
                                                              C.byref(cfg), _stream(stream)))


def gabsplat_batch_status_copy(frame, dst_ptr, stream=None):
    _check("gabsplat_batch_status_copy", lib.gabsplat_batch_status_copy(C.byref(frame), C.c_void_p(dst_ptr),
                                                                        _stream(stream)))


def gabsplat_batch_graph_create(frame, cfg, stream=None):
    g = C.c_void_p()
    _check("gabsplat_batch_graph_create", lib.gabsplat_batch_graph_create(C.byref(frame), C.byref(cfg),
                                                                          _stream(stream), C.byref(g)))
    return g


def gabsplat_batch_graph_launch(graph, views, stream=None):
    _check("gabsplat_batch_graph_launch", lib.gabsplat_batch_graph_launch(graph, _view_array(views), len(views),
                                                                          _stream(stream)))


def gabsplat_batch_graph_destroy(graph):
    lib.gabsplat_batch_graph_destroy(graph)


def make_view(prims: "gs_prims", cam: "gs_camera", out_rgb, out_T=None) -> "gs_view":
    v = gs_view()
    v.prims, v.cam = prims, cam
    v.out_rgb = out_rgb.data_ptr()
    v.out_T = out_T.data_ptr() if out_T is not None else None
    return v


def status_string(st):
    return lib.gabsplat_status_string(int(st)).decode()


def gabsplat_status_string(st):
    return status_string(st)


def gabsplat_version():
    return lib.gabsplat_version().decode()


# ---- struct builders ------------------------------------------------------------------------
def make_camera(cam: dict) -> gs_camera:
    c = gs_camera()
    R = np.asarray(cam["R"], np.float32).reshape(9)
    t = np.asarray(cam["t"], np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.znear, c.zfar = cam["znear"], cam["zfar"]
    return c


def make_config(eps2d=0.3, alpha_max=0.99, alpha_min=1.0 / 255.0, T_min=1e-4, bg=(0.0, 0.0, 0.0),
                flags=0) -> gs_config:
    g = gs_config()
    g.eps2d, g.alpha_max, g.alpha_min, g.T_min = eps2d, alpha_max, alpha_min, T_min
    for i in range(3):
        g.bg[i] = float(bg[i])
    g.flags = flags
    return g


def make_prims(t: dict, storage=GS_F32) -> gs_prims:
    """t: dict of contiguous CUDA tensors (means, scales, quats, opacity, sh, freqs, weights)."""
    p = gs_prims()
    n = t["means"].shape[0]
    K = t["weights"].shape[1] if t.get("weights") is not None else 0
    p.n, p.K = n, K
    p.sh_degree = int(round(t["sh"].shape[1] ** 0.5)) - 1
    p.storage = storage
    for k in ("means", "scales", "quats", "opacity", "sh"):
        setattr(p, k, t[k].data_ptr())
    p.freqs = t["freqs"].data_ptr() if K > 0 else None
    p.weights = t["weights"].data_ptr() if K > 0 else None
    return p


def make_densify_config(grad_threshold=2e-4, dense_scale=0.05, min_opacity=0.01, max_scale=0.0, split_divisor=1.6,
                        child_freq=1e-3, child_weight=1e-2) -> gs_densify_config:
    c = gs_densify_config()
    c.grad_threshold, c.dense_scale, c.min_opacity, c.max_scale = grad_threshold, dense_scale, min_opacity, max_scale
    c.split_divisor, c.child_freq, c.child_weight = split_divisor, child_freq, child_weight
    return c


def make_prim_arrays(t: dict) -> gs_prim_arrays:
    """Writable arrays from a dict of contiguous CUDA tensors (means, scales, quats, opacity, sh, freqs, weights)."""
    a = gs_prim_arrays()
    for k in ("means", "scales", "quats", "opacity", "sh", "freqs", "weights"):
        v = t.get(k)
        setattr(a, k, v.data_ptr() if v is not None and v.numel() > 0 else None)
    return a


def gabsplat_densify_accumulate(frame, means2d_grad, grad_accum, denom, stream=None):
    _check("gabsplat_densify_accumulate", lib.gabsplat_densify_accumulate(
        C.byref(frame), _ptr(means2d_grad), _ptr(grad_accum), _ptr(denom), _stream(stream)))


def gabsplat_densify_scratch_bytes(n):
    return int(lib.gabsplat_densify_scratch_bytes(n))


def gabsplat_densify(prims, grad_accum, denom, split_noise, cfg, out, out_capacity, counts, scratch, stream=None):
    """prims: gs_prims; out: gs_prim_arrays with room for out_capacity (>= 2 n) rows; counts: int32[4] on the device."""
    _check("gabsplat_densify", lib.gabsplat_densify(C.byref(prims), _ptr(grad_accum), _ptr(denom), _ptr(split_noise),
                                                    C.byref(cfg), C.byref(out), out_capacity, _ptr(counts),
                                                    _ptr(scratch), _stream(stream)))


def gabsplat_reset_opacity_weights(arrays, n, K, storage, opacity_cap=0.02, weight=0.01, stream=None):
    _check("gabsplat_reset_opacity_weights", lib.gabsplat_reset_opacity_weights(
        C.byref(arrays), n, K, storage, opacity_cap, weight, _stream(stream)))

"""Thin Python binding of libgs.so (include/gs.h), through ctypes.

Argument marshalling only: every step runs in the library's CUDA kernels.
Tensors are torch CUDA tensors; their device pointers and the current CUDA
stream are handed to the C ABI.  If the library is missing or cannot be
loaded, importing the binding raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

_lib = None

GS_OK, GS_EINVAL, GS_ENOMEM, GS_ECUDA, GS_ECAPACITY, GS_ETIMEOUT, GS_EBUSY, GS_EAGAIN, GS_ESTATE = range(9)
_NAMES = ["GS_OK", "GS_EINVAL", "GS_ENOMEM", "GS_ECUDA", "GS_ECAPACITY", "GS_ETIMEOUT", "GS_EBUSY",
          "GS_EAGAIN", "GS_ESTATE"]

(GS_BUF_REC0, GS_BUF_REC1, GS_BUF_REC2, GS_BUF_KEYS, GS_BUF_VALS, GS_BUF_RANGES, GS_BUF_TFINAL,
 GS_BUF_NLAST, GS_BUF_G2D, GS_BUF_REC3, GS_BUF_SORT_CTRL, GS_BUF_VISMASK, GS_BUF_DEPTH_CTRL) = range(13)
LOG2E = 1.4426950408889634


class GsError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (_NAMES[status] if 0 <= status < len(_NAMES) else status, msg))


class gs_config(ctypes.Structure):
    _fields_ = [("max_gaussians", ctypes.c_int64), ("max_views", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("instance_capacity", ctypes.c_int64)]


class gs_camera(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 16), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("znear", ctypes.c_float), ("bg", ctypes.c_float * 3)]


class gs_params(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n", ctypes.c_int64), ("stride", ctypes.c_int64),
                ("sh_degree", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class gs_adam_hp(ctypes.Structure):
    _fields_ = [("lr_mean", ctypes.c_float), ("lr_scale", ctypes.c_float), ("lr_quat", ctypes.c_float),
                ("lr_opacity", ctypes.c_float), ("lr_sh_dc", ctypes.c_float), ("lr_sh_rest", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("flags", ctypes.c_int32)]


GS_ADAM_SQRT_BATCH_LR = 1
GS_ADAM_VISIBLE_ONLY = 2


def adam_hp_struct(hp: dict) -> gs_adam_hp:
    """hp: lr_mean, lr_scale, lr_quat, lr_opacity, lr_sh_dc, lr_sh_rest, and
    optionally beta1, beta2, eps, sqrt_batch_lr (scale the rates by
    sqrt(views per batch)) and visible_only (the sparse, visible-only step)."""
    flags = (GS_ADAM_SQRT_BATCH_LR if hp.get("sqrt_batch_lr", False) else 0) | \
        (GS_ADAM_VISIBLE_ONLY if hp.get("visible_only", False) else 0)
    return gs_adam_hp(hp["lr_mean"], hp["lr_scale"], hp["lr_quat"], hp["lr_opacity"], hp["lr_sh_dc"],
                      hp["lr_sh_rest"], hp.get("beta1", 0.9), hp.get("beta2", 0.999), hp.get("eps", 1e-15),
                      flags)


class gs_densify_hp(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("percent_dense", ctypes.c_float),
                ("scene_extent", ctypes.c_float), ("min_opacity", ctypes.c_float), ("split_n", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class gs_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


GS_OPT_RASTER_FWD, GS_OPT_RASTER_BWD, GS_OPT_BWD_DIRECT, GS_OPT_SORT_ITEMS, GS_OPT_SORT_WAIT, GS_OPT_TILE_ORDER = \
    0, 1, 2, 3, 4, 5

class gs_serve_cfg(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch_views", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("max_view_pixels", ctypes.c_int32), ("memory_budget_bytes", ctypes.c_int64),
                ("output_pool_bytes", ctypes.c_int64)]


EXPORTS = ["gs_raster_fwd_l1", "gs_train_graph_capture", "gs_train_graph_launch", "gs_train_graph_launch_host", "gs_serve_create", "gs_serve_destroy", "gs_serve_submit", "gs_serve_poll", "gs_serve_release",
           "gs_serve_stats", "gs_set_option", "gs_get_option", "gs_l1_loss_noalloc", "gs_profile_enable", "gs_profile_read", "gs_profile_reset", "gs_create", "gs_destroy", "gs_last_error", "gs_set_stream", "gs_sync", "gs_project",
           "gs_bin_sort", "gs_raster_fwd", "gs_raster_bwd", "gs_l1_loss", "gs_adam", "gs_get_buffer",
           "gs_get_counts", "gs_pair_stats", "gs_serve_timeline", "gs_ssim_loss",
           "gs_image_metrics", "gs_iso_crossings", "gs_init_gaussians",
           "gs_set_densify_stats", "gs_densify"]


def load(path: str | None = None):
    """Load libgs.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    L = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    L.gs_create.argtypes = [P(vp), ctypes.c_int, P(gs_config)]
    L.gs_destroy.argtypes = [vp]
    L.gs_destroy.restype = None
    L.gs_last_error.argtypes = [vp]
    L.gs_last_error.restype = ctypes.c_char_p
    L.gs_set_stream.argtypes = [vp, vp]
    L.gs_sync.argtypes = [vp]
    L.gs_project.argtypes = [vp, P(gs_params), P(gs_camera), i32]
    L.gs_bin_sort.argtypes = [vp]
    L.gs_raster_fwd.argtypes = [vp, vp]
    L.gs_raster_bwd.argtypes = [vp, P(gs_params), vp, P(gs_params)]
    L.gs_l1_loss.argtypes = [vp, vp, vp, i64, vp, vp]
    L.gs_adam.argtypes = [vp, P(gs_params), P(gs_params), P(gs_params), P(gs_params), P(gs_adam_hp), i64]
    L.gs_get_buffer.argtypes = [vp, i32, P(vp), P(i64)]
    L.gs_get_counts.argtypes = [vp, P(i64), P(i64), P(i64)]
    L.gs_train_graph_capture.argtypes = [vp, P(gs_params), P(gs_params), P(gs_params), P(gs_params), P(gs_adam_hp),
                                         P(gs_camera), i32, vp, vp, vp, vp]
    L.gs_raster_fwd_l1.argtypes = [vp, vp, vp, vp, vp]
    L.gs_train_graph_launch.argtypes = [vp, P(gs_camera), i32, vp, i64]
    L.gs_train_graph_launch_host.argtypes = [vp, P(gs_camera), i32, vp, i64, vp]
    L.gs_serve_create.argtypes = [P(vp), ctypes.c_int, P(gs_params), P(gs_serve_cfg)]
    L.gs_serve_destroy.argtypes = [vp]
    L.gs_serve_destroy.restype = None
    L.gs_serve_submit.argtypes = [vp, P(gs_camera), vp, P(ctypes.c_uint64)]
    L.gs_serve_poll.argtypes = [vp, ctypes.c_uint64, i64, P(vp), P(ctypes.c_int)]
    L.gs_serve_release.argtypes = [vp, ctypes.c_uint64]
    L.gs_serve_stats.argtypes = [vp, P(i64), P(i64), P(i64)]
    L.gs_set_option.argtypes = [vp, i32, i64]
    L.gs_get_option.argtypes = [vp, i32, P(i64)]
    L.gs_l1_loss_noalloc.argtypes = [vp, vp, i64, vp, vp, vp]
    L.gs_profile_enable.argtypes = [vp, i32]
    L.gs_profile_read.argtypes = [vp, P(gs_kernel_stat), i32, P(i32)]
    L.gs_profile_reset.argtypes = [vp]
    L.gs_pair_stats.argtypes = [vp, P(i64), P(i64)]
    L.gs_ssim_loss.argtypes = [vp, vp, vp, ctypes.c_float, vp, vp]
    L.gs_set_densify_stats.argtypes = [vp, vp, vp]
    L.gs_densify.argtypes = [vp, P(gs_params), P(gs_params), P(gs_params), vp, vp, vp, P(gs_densify_hp),
                             P(gs_params), P(gs_params), P(gs_params), P(i64)]
    L.gs_iso_crossings.argtypes = [vp, vp, i32, i32, i32, ctypes.c_float, P(ctypes.c_float), P(ctypes.c_float),
                                   vp, vp, i64, P(i64)]
    L.gs_init_gaussians.argtypes = [vp, vp, vp, i64, vp, i64, ctypes.c_float, ctypes.c_float, P(gs_params)]
    L.gs_image_metrics.argtypes = [vp, vp, vp, P(ctypes.c_double), P(ctypes.c_double)]
    L.gs_serve_timeline.argtypes = [vp, P(ctypes.c_double), i32, P(i32), P(i64)]
    for name in EXPORTS:
        f = getattr(L, name)
        if f.restype is ctypes.c_int:
            f.restype = ctypes.c_int
    _lib = L
    return L


def camera_struct(cam) -> gs_camera:
    c = gs_camera()
    vm = np.asarray(cam["viewmat"], np.float64).reshape(16)
    for i in range(16):
        c.viewmat[i] = float(vm[i])
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.znear = float(cam["znear"])
    for i in range(3):
        c.bg[i] = float(cam["bg"][i])
    return c


def params_struct(t: torch.Tensor, n: int, deg: int) -> gs_params:
    if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.is_contiguous()):
        raise ValueError("parameters must be a contiguous float32 CUDA tensor [P, stride]")
    if t.shape[0] != 11 + 3 * (deg + 1) ** 2:
        raise ValueError("plane count %d does not match SH degree %d" % (t.shape[0], deg))
    return gs_params(t.data_ptr(), n, t.shape[1], deg, 0)


class _DevArray:
    """Zero-copy view of a device buffer for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr, strides=None):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": strides}


class Context:
    """One gs_ctx.  Methods are the C ABI's calls with tensor arguments."""

    def __init__(self, device: int = 0, max_views: int = 64, instance_capacity: int = 0):
        self.L = load()
        self.device = device
        cfg = gs_config(0, max_views, 0, instance_capacity)
        h = ctypes.c_void_p()
        st = self.L.gs_create(ctypes.byref(h), device, ctypes.byref(cfg))
        if st != GS_OK:
            raise GsError(st, "gs_create(device=%d) failed" % device)
        self.h = h
        self._stream = None

    def close(self):
        if getattr(self, "h", None):
            self.L.gs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != GS_OK:
            raise GsError(st, "%s: %s" % (what, self.L.gs_last_error(self.h).decode()))

    def _bind_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            self._check(self.L.gs_set_stream(self.h, ctypes.c_void_p(s)), "gs_set_stream")
            self._stream = s

    # -- the path ---------------------------------------------------------
    def gs_project(self, params: torch.Tensor, n: int, deg: int, cams):
        self._bind_stream()
        p = params_struct(params, n, deg)
        arr = (gs_camera * len(cams))(*[camera_struct(c) for c in cams])
        self._check(self.L.gs_project(self.h, ctypes.byref(p), arr, len(cams)), "gs_project")

    def gs_bin_sort(self):
        self._bind_stream()
        self._check(self.L.gs_bin_sort(self.h), "gs_bin_sort")

    def gs_raster_fwd(self, images: torch.Tensor):
        self._bind_stream()
        assert images.is_cuda and images.dtype == torch.float32 and images.is_contiguous()
        self._check(self.L.gs_raster_fwd(self.h, ctypes.c_void_p(images.data_ptr())), "gs_raster_fwd")

    def gs_raster_fwd_l1(self, images, targets: torch.Tensor, loss: torch.Tensor, dimages: torch.Tensor):
        """Forward compositing fused with the L1 loss (images may be None)."""
        self._bind_stream()
        for t in (targets, loss, dimages):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        ip = ctypes.c_void_p(images.data_ptr()) if images is not None else None
        self._check(self.L.gs_raster_fwd_l1(self.h, ip, ctypes.c_void_p(targets.data_ptr()),
                                            ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(dimages.data_ptr())),
                    "gs_raster_fwd_l1")

    def gs_raster_bwd(self, params: torch.Tensor, n: int, deg: int, dL_dimages: torch.Tensor,
                      grads: torch.Tensor):
        self._bind_stream()
        assert dL_dimages.is_cuda and dL_dimages.dtype == torch.float32 and dL_dimages.is_contiguous()
        p = params_struct(params, n, deg)
        g = params_struct(grads, n, deg)
        self._check(self.L.gs_raster_bwd(self.h, ctypes.byref(p), ctypes.c_void_p(dL_dimages.data_ptr()),
                                         ctypes.byref(g)), "gs_raster_bwd")

    def gs_l1_loss(self, x: torch.Tensor, y: torch.Tensor, loss: torch.Tensor | None, grad: torch.Tensor | None):
        self._bind_stream()
        assert x.is_contiguous() and y.is_contiguous() and x.numel() == y.numel()
        self._check(self.L.gs_l1_loss(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      x.numel(), ctypes.c_void_p(loss.data_ptr() if loss is not None else 0),
                                      ctypes.c_void_p(grad.data_ptr() if grad is not None else 0)), "gs_l1_loss")

    def gs_adam(self, p, g, m, v, n, deg, hp: dict, step: int):
        self._bind_stream()
        sp, sg, sm, sv = (params_struct(t, n, deg) for t in (p, g, m, v))
        h = adam_hp_struct(hp)
        self._check(self.L.gs_adam(self.h, ctypes.byref(sp), ctypes.byref(sg), ctypes.byref(sm), ctypes.byref(sv),
                                   ctypes.byref(h), int(step)), "gs_adam")

    def gs_train_graph_capture(self, p, g, m, v, n, deg, hp: dict, cams, targets, images, dimages, loss):
        """Capture one training step (needs instance_capacity > 0).  Keep every
        tensor alive and in place while the graph is used."""
        self._bind_stream()
        sp, sg, sm, sv = (params_struct(t, n, deg) for t in (p, g, m, v))
        h = adam_hp_struct(hp)
        arr = (gs_camera * len(cams))(*[camera_struct(c) for c in cams])
        self._graph_keep = (sp, sg, sm, sv, h, p, g, m, v, targets, images, dimages, loss)
        self._check(self.L.gs_train_graph_capture(
            self.h, ctypes.byref(sp), ctypes.byref(sg), ctypes.byref(sm), ctypes.byref(sv), ctypes.byref(h), arr,
            len(cams), ctypes.c_void_p(targets.data_ptr()), ctypes.c_void_p(images.data_ptr()),
            ctypes.c_void_p(dimages.data_ptr()), ctypes.c_void_p(loss.data_ptr())), "gs_train_graph_capture")

    def gs_train_graph_launch(self, cams, targets: torch.Tensor, step: int):
        self._bind_stream()
        arr = (gs_camera * len(cams))(*[camera_struct(c) for c in cams])
        self._check(self.L.gs_train_graph_launch(self.h, arr, len(cams), ctypes.c_void_p(targets.data_ptr()),
                                                 int(step)), "gs_train_graph_launch")

    def gs_train_graph_launch_host(self, cams, host_targets: torch.Tensor, step: int, host_loss=None):
        """Replay with targets in host memory (pinned for overlap) and the loss
        read back into `host_loss` (a 1-element CPU float32 tensor, or None).
        Keep both alive and unchanged until gs_sync."""
        self._bind_stream()
        assert host_targets.device.type == "cpu" and host_targets.dtype == torch.float32
        assert host_targets.is_contiguous()
        lp = None
        if host_loss is not None:
            assert host_loss.device.type == "cpu" and host_loss.dtype == torch.float32
            lp = ctypes.c_void_p(host_loss.data_ptr())
        arr = (gs_camera * len(cams))(*[camera_struct(c) for c in cams])
        self._check(self.L.gs_train_graph_launch_host(self.h, arr, len(cams), ctypes.c_void_p(host_targets.data_ptr()),
                                                      int(step), lp), "gs_train_graph_launch_host")

    def gs_ssim_loss(self, images: torch.Tensor, targets: torch.Tensor, lam: float, loss=None, dimages=None):
        """(1 - lam) L1 + lam (1 - SSIM) over the last projected batch's views."""
        self._bind_stream()
        for t in (images, targets):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        self._check(self.L.gs_ssim_loss(self.h, ctypes.c_void_p(images.data_ptr()), ctypes.c_void_p(targets.data_ptr()),
                                        float(lam), ctypes.c_void_p(loss.data_ptr() if loss is not None else 0),
                                        ctypes.c_void_p(dimages.data_ptr() if dimages is not None else 0)),
                    "gs_ssim_loss")

    def gs_image_metrics(self, images: torch.Tensor, targets: torch.Tensor, views: int):
        """(SSIM per view, PSNR per view) of the last projected batch."""
        self._bind_stream()
        s = (ctypes.c_double * views)()
        p = (ctypes.c_double * views)()
        self._check(self.L.gs_image_metrics(self.h, ctypes.c_void_p(images.data_ptr()),
                                            ctypes.c_void_p(targets.data_ptr()), s, p), "gs_image_metrics")
        return list(s), list(p)

    def gs_iso_crossings(self, volume: torch.Tensor, iso: float, origin, spacing):
        """(points [m, 3], normals [m, 3]) device tensors of the level's edge
        crossings of a [nz, ny, nx] float32 CUDA volume."""
        self._bind_stream()
        assert volume.is_cuda and volume.dtype == torch.float32 and volume.is_contiguous() and volume.dim() == 3
        nz, ny, nx = volume.shape
        o = (ctypes.c_float * 3)(*[float(x) for x in origin])
        h = (ctypes.c_float * 3)(*[float(x) for x in spacing])
        cnt = ctypes.c_int64()
        self._check(self.L.gs_iso_crossings(self.h, ctypes.c_void_p(volume.data_ptr()), nx, ny, nz, float(iso), o, h,
                                            None, None, 0, ctypes.byref(cnt)), "gs_iso_crossings")
        m = cnt.value
        pts = torch.empty((max(m, 1), 3), device=volume.device, dtype=torch.float32)
        nrm = torch.empty_like(pts)
        self._check(self.L.gs_iso_crossings(self.h, ctypes.c_void_p(volume.data_ptr()), nx, ny, nz, float(iso), o, h,
                                            ctypes.c_void_p(pts.data_ptr()), ctypes.c_void_p(nrm.data_ptr()), m,
                                            ctypes.byref(cnt)), "gs_iso_crossings")
        return pts[:m], nrm[:m]

    def gs_init_gaussians(self, points: torch.Tensor, normals: torch.Tensor, out: torch.Tensor, n: int, deg: int,
                          select: torch.Tensor | None = None, flatten: float = 0.3, opacity_logit: float = 2.0):
        """Write the initial Gaussians (plane layout) of the selected points into `out`."""
        self._bind_stream()
        for t in (points, normals):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.shape[1:] == (3,)
        sp = None
        if select is not None:
            assert select.is_cuda and select.dtype == torch.int64 and select.is_contiguous()
            sp = ctypes.c_void_p(select.data_ptr())
        o = params_struct(out, n, deg)
        self._check(self.L.gs_init_gaussians(self.h, ctypes.c_void_p(points.data_ptr()),
                                             ctypes.c_void_p(normals.data_ptr()), points.shape[0], sp, n,
                                             float(flatten), float(opacity_logit), ctypes.byref(o)),
                    "gs_init_gaussians")

    def gs_set_densify_stats(self, grad_accum, count):
        """Accumulate the densification statistic into these float32 CUDA
        tensors in every following gs_raster_bwd (None, None: stop)."""
        ga = ctypes.c_void_p(grad_accum.data_ptr()) if grad_accum is not None else None
        ct = ctypes.c_void_p(count.data_ptr()) if count is not None else None
        self._keep_stats = (grad_accum, count)
        self._check(self.L.gs_set_densify_stats(self.h, ga, ct), "gs_set_densify_stats")

    def gs_densify(self, p, m, v, n, deg, grad_accum, count, noise, hp: dict, p_out, m_out, v_out) -> int:
        """One densification step into the output tensors; returns the new size."""
        self._bind_stream()
        sp, sm, sv = (params_struct(t, n, deg) for t in (p, m, v))
        so, smo, svo = (gs_params(t.data_ptr(), 1, t.shape[1], deg, 0) for t in (p_out, m_out, v_out))
        h = gs_densify_hp(hp.get("grad_threshold", 2e-4), hp.get("percent_dense", 0.01), hp["scene_extent"],
                          hp.get("min_opacity", 0.005), hp.get("split_n", 2), 0)
        nout = ctypes.c_int64()
        st = self.L.gs_densify(self.h, ctypes.byref(sp), ctypes.byref(sm), ctypes.byref(sv),
                               ctypes.c_void_p(grad_accum.data_ptr()), ctypes.c_void_p(count.data_ptr()),
                               ctypes.c_void_p(noise.data_ptr()), ctypes.byref(h), ctypes.byref(so),
                               ctypes.byref(smo), ctypes.byref(svo), ctypes.byref(nout))
        if st != GS_OK:
            e = GsError(st, "gs_densify: %s" % self.L.gs_last_error(self.h).decode())
            e.n_out = nout.value
            raise e
        return nout.value

    def gs_sync(self):
        self._check(self.L.gs_sync(self.h), "gs_sync")

    # -- options ----------------------------------------------------------
    def gs_set_option(self, option: int, value: int):
        self._check(self.L.gs_set_option(self.h, option, int(value)), "gs_set_option")

    def gs_get_option(self, option: int) -> int:
        v = ctypes.c_int64()
        self._check(self.L.gs_get_option(self.h, option, ctypes.byref(v)), "gs_get_option")
        return v.value

    # -- profiling --------------------------------------------------------
    def profile_enable(self, on: bool = True):
        self._check(self.L.gs_profile_enable(self.h, 1 if on else 0), "gs_profile_enable")

    def profile_reset(self):
        self._check(self.L.gs_profile_reset(self.h), "gs_profile_reset")

    def profile_read(self):
        arr = (gs_kernel_stat * 64)()
        cnt = ctypes.c_int32()
        self._check(self.L.gs_profile_read(self.h, arr, 64, ctypes.byref(cnt)), "gs_profile_read")
        return [{"name": arr[i].name.decode(), "launches": int(arr[i].launches), "total_ms": float(arr[i].total_ms)}
                for i in range(min(cnt.value, 64))]

    # -- inspection -------------------------------------------------------
    def gs_get_counts(self):
        i, b, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.L.gs_get_counts(self.h, ctypes.byref(i), ctypes.byref(b), ctypes.byref(p)),
                    "gs_get_counts")
        return i.value, b.value, p.value

    def gs_pair_stats(self):
        """(list entries up to each pixel's last contributor, contributing
        pairs) of the last forward pass."""
        self._bind_stream()
        e, c = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.L.gs_pair_stats(self.h, ctypes.byref(e), ctypes.byref(c)), "gs_pair_stats")
        return e.value, c.value

    def gs_get_buffer(self, which: int) -> torch.Tensor:
        """Copy of an intermediate buffer as a torch tensor."""
        ptr, cnt = ctypes.c_void_p(), ctypes.c_int64()
        self._check(self.L.gs_get_buffer(self.h, which, ctypes.byref(ptr), ctypes.byref(cnt)), "gs_get_buffer")
        n = cnt.value
        spec = {GS_BUF_REC0: ((n, 4), "<f4"), GS_BUF_REC1: ((n, 4), "<f4"), GS_BUF_REC2: ((n, 4), "<f4"),
                GS_BUF_KEYS: ((n,), "<i4"), GS_BUF_VALS: ((n,), "<i4"), GS_BUF_RANGES: ((n, 2), "<i4"),
                GS_BUF_TFINAL: ((n,), "<f4"), GS_BUF_NLAST: ((n,), "<i4"), GS_BUF_G2D: ((n,), "<f4"), GS_BUF_REC3: ((n, 4), "<i4"),
                GS_BUF_SORT_CTRL: ((n,), "<i4"), GS_BUF_VISMASK: ((n,), "<i8"),
                GS_BUF_DEPTH_CTRL: ((n,), "<i4")}[which]
        if n == 0:
            return torch.empty(spec[0], device="cuda:%d" % self.device,
                               dtype={"<f4": torch.float32, "<i8": torch.int64, "<i4": torch.int32}[spec[1]])
        # the three projected records are interleaved (48 bytes per entry)
        strides = (48, 4) if which in (GS_BUF_REC0, GS_BUF_REC1, GS_BUF_REC2) else None
        t = torch.as_tensor(_DevArray(ptr.value, *spec, strides=strides), device="cuda:%d" % self.device)
        return t.clone()


def gs_l1_loss_noalloc(x: torch.Tensor, y: torch.Tensor, loss: torch.Tensor | None,
                       grad: torch.Tensor | None):
    """L1 loss through the allocation-free entry point (no context needed):
    for callers that may not allocate device memory.  Runs on x's device and
    the current stream; raises GsError on a non-OK status."""
    L = load()
    assert x.is_cuda and x.is_contiguous() and y.is_contiguous() and x.numel() == y.numel()
    with torch.cuda.device(x.device):
        s = torch.cuda.current_stream(x.device).cuda_stream
        st = L.gs_l1_loss_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(),
                                  ctypes.c_void_p(loss.data_ptr() if loss is not None else 0),
                                  ctypes.c_void_p(grad.data_ptr() if grad is not None else 0), ctypes.c_void_p(s))
    if st != GS_OK:
        raise GsError(st, "gs_l1_loss_noalloc(count=%d)" % x.numel())


class Server:
    """Continuous-batching render server (gs_serve_*): the resident parameter
    tensor must stay alive and unchanged while the server runs."""

    def __init__(self, params: torch.Tensor, n: int, deg: int, device: int = 0, slots: int = 2,
                 max_batch_views: int = 16, max_queue: int = 4096, memory_budget_bytes: int = 16 << 30,
                 output_pool_bytes: int = 1 << 30, max_view_pixels: int = 0):
        self.L = load()
        self.params = params  # keep alive
        self.device = device
        p = params_struct(params, n, deg)
        cfg = gs_serve_cfg(slots, max_batch_views, max_queue, max_view_pixels, memory_budget_bytes,
                           output_pool_bytes)
        h = ctypes.c_void_p()
        st = self.L.gs_serve_create(ctypes.byref(h), device, ctypes.byref(p), ctypes.byref(cfg))
        if st != GS_OK:
            raise GsError(st, "gs_serve_create failed")
        self.h = h
        self._shape = {}

    def close(self):
        if getattr(self, "h", None):
            self.L.gs_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def gs_serve_submit(self, cam, out: torch.Tensor | None = None) -> int:
        c = camera_struct(cam)
        t = ctypes.c_uint64()
        st = self.L.gs_serve_submit(self.h, ctypes.byref(c), ctypes.c_void_p(out.data_ptr() if out is not None else 0),
                                    ctypes.byref(t))
        if st != GS_OK:
            raise GsError(st, "gs_serve_submit")
        self._shape[t.value] = (3, int(cam["height"]), int(cam["width"]))
        return t.value

    def gs_serve_poll(self, ticket: int, timeout_us: int = -1):
        """Returns (status, image view or None); status GS_EAGAIN on timeout."""
        ptr, res = ctypes.c_void_p(), ctypes.c_int()
        st = self.L.gs_serve_poll(self.h, ticket, int(timeout_us),
                                  ctypes.byref(ptr), ctypes.byref(res))
        if st == GS_EAGAIN:
            return GS_EAGAIN, None
        if st != GS_OK:
            raise GsError(st, "gs_serve_poll(%d)" % ticket)
        if res.value != GS_OK:
            return res.value, None
        img = torch.as_tensor(_DevArray(ptr.value, self._shape[ticket], "<f4"), device="cuda:%d" % self.device)
        return GS_OK, img

    def gs_serve_release(self, ticket: int):
        st = self.L.gs_serve_release(self.h, ticket)
        self._shape.pop(ticket, None)
        if st != GS_OK:
            raise GsError(st, "gs_serve_release(%d)" % ticket)

    def gs_serve_timeline(self, cap: int = 4096):
        """((start_ms, end_ms) of the most recent retired batches on the
        device timeline, oldest first; batches rendered again after a
        capacity overflow)."""
        buf = (ctypes.c_double * (2 * cap))()
        cnt, retried = ctypes.c_int32(), ctypes.c_int64()
        st = self.L.gs_serve_timeline(self.h, buf, cap, ctypes.byref(cnt), ctypes.byref(retried))
        if st != GS_OK:
            raise GsError(st, "gs_serve_timeline")
        return [(buf[2 * i], buf[2 * i + 1]) for i in range(cnt.value)], retried.value

    def gs_serve_stats(self):
        b, r, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self.L.gs_serve_stats(self.h, ctypes.byref(b), ctypes.byref(r), ctypes.byref(p))
        return {"batches": b.value, "rendered": r.value, "pending": p.value}


def image_offsets(cams):
    """Start (in floats) of each view's [3][H][W] block in a batch image buffer."""
    offs, o = [], 0
    for c in cams:
        offs.append(o)
        o += 3 * c["width"] * c["height"]
    return offs, o


def split_images(buf: torch.Tensor, cams):
    offs, _ = image_offsets(cams)
    return [buf[o:o + 3 * c["width"] * c["height"]].view(3, c["height"], c["width"]) for o, c in zip(offs, cams)]

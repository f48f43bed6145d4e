"""Python access to the FP64 CPU oracle (gs_oracle.c) through ctypes.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg import this module.  The product path never does.

All arrays handed to the oracle are float64 copies of the float32 inputs, so
the oracle sees exactly the values the CUDA path sees.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgs_oracle.so")
_lock = threading.Lock()
_lib = None

CAM_LEN = 26
# Gaussian flags (mirrors the enum in gs_oracle.c)
G_VISIBLE, G_MARG_ZNEAR, G_MARG_RECT, G_MARG_GUARD, G_MARG_SHCLAMP = 1, 2, 4, 8, 16
G_MARG_ANY_GRAD = G_MARG_ZNEAR | G_MARG_RECT | G_MARG_GUARD | G_MARG_SHCLAMP


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into oracle/_build/libgs_oracle.so (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            up = ctypes.POINTER(ctypes.c_uint8)
            cl, ci = ctypes.c_long, ctypes.c_int
            L.or_project.argtypes = [dp, cl, cl, ci, dp, dp, ip]
            L.or_render.argtypes = [dp, cl, cl, ci, dp, up, dp, dp, up]
            L.or_render.restype = cl
            L.or_render_pixels.argtypes = [dp, cl, cl, ci, dp, cl, ip, ip, dp, dp, up]
            L.or_render_grad.argtypes = [dp, cl, cl, ci, dp, ci, dp, dp, dp]
            L.or_project_jacobian.argtypes = [dp, cl, cl, ci, dp, cl, dp]
            L.or_project_jacobian.restype = ci
            L.or_gaussian_flags.argtypes = [dp, cl, cl, ci, dp, ip]
            L.or_l1.argtypes = [dp, dp, cl, dp]
            L.or_l1.restype = ctypes.c_double
            L.or_adam.argtypes = [dp, dp, dp, dp, ci, cl, cl, dp, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, cl]
            L.or_adam_visible.argtypes = [dp, dp, dp, dp, ci, cl, cl, dp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, cl, up]
            L.or_sh_basis.argtypes = [ci, dp, cl, dp]
            L.or_num_threads.restype = ci
            _lib = L
    return _lib


def _p(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def cam_record(cam) -> np.ndarray:
    r = np.zeros(CAM_LEN)
    r[0:16] = np.asarray(cam["viewmat"], np.float64).reshape(16)
    r[16:20] = [cam["fx"], cam["fy"], cam["cx"], cam["cy"]]
    r[20:22] = [cam["width"], cam["height"]]
    r[22] = cam["znear"]
    r[23:26] = cam["bg"]
    return r


def _params64(scene):
    p = np.ascontiguousarray(scene["params"], dtype=np.float64)
    return p, p.shape[1]


def num_threads() -> int:
    return int(lib().or_num_threads())


def project(scene, cam):
    """Per-Gaussian projection: dict of float64 / int arrays."""
    p, stride = _params64(scene)
    n = scene["n"]
    f = np.zeros((n, 16))
    i = np.zeros((n, 8), dtype=np.int32)
    c = cam_record(cam)
    lib().or_project(_p(p), n, stride, scene["deg"], _p(c), _p(f), _p(i, ctypes.c_int))
    return {"mean2d": f[:, 0:2], "depth": f[:, 2], "conic": f[:, 3:6], "opacity": f[:, 6],
            "rgb": f[:, 7:10], "ext": f[:, 10], "raw_rgb": f[:, 11:14], "flags": i[:, 0],
            "radius": i[:, 1], "rect": i[:, 2:6], "tiles": i[:, 6]}


def render(scene, cam, tile_want=None):
    """Image [3,H,W], T_final [H,W], marginal mask [H,W] (bool), pairs composited."""
    p, stride = _params64(scene)
    W, H = cam["width"], cam["height"]
    img = np.zeros((3, H, W))
    tf = np.zeros((H, W))
    mg = np.zeros((H, W), dtype=np.uint8)
    c = cam_record(cam)
    want = None
    if tile_want is not None:
        want = np.ascontiguousarray(tile_want, dtype=np.uint8)
    pairs = lib().or_render(_p(p), scene["n"], stride, scene["deg"], _p(c),
                            None if want is None else _p(want, ctypes.c_uint8),
                            _p(img), _p(tf), _p(mg, ctypes.c_uint8))
    return img, tf, mg.astype(bool), int(pairs)


def render_pixels(scene, cam, xs, ys):
    p, stride = _params64(scene)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    m = xs.shape[0]
    rgb = np.zeros((m, 3))
    t = np.zeros(m)
    mg = np.zeros(m, dtype=np.uint8)
    c = cam_record(cam)
    lib().or_render_pixels(_p(p), scene["n"], stride, scene["deg"], _p(c), m,
                           _p(xs, ctypes.c_int), _p(ys, ctypes.c_int), _p(rgb), _p(t),
                           _p(mg, ctypes.c_uint8))
    return rgb, t, mg.astype(bool)


def render_grad(scene, cams, dimgs, want_2d=False):
    """Gradient of sum_v <dimgs[v], image_v> w.r.t. the [P, stride] parameters.

    dimgs: list of [3,H,W] arrays (one per camera).  Returns grad (float64
    [P, stride]) and, if want_2d, the per-view 2D gradients [B, n, 9]
    (mu_x, mu_y, A, B, C, sigma, r, g, b)."""
    p, stride = _params64(scene)
    n = scene["n"]
    B = len(cams)
    cr = np.concatenate([cam_record(c) for c in cams])
    d = np.concatenate([np.ascontiguousarray(x, dtype=np.float64).ravel() for x in dimgs])
    grad = np.zeros_like(p)
    g2d = np.zeros((B, n, 9)) if want_2d else None
    lib().or_render_grad(_p(p), n, stride, scene["deg"], _p(cr), B, _p(d), _p(grad),
                         None if g2d is None else _p(g2d))
    return (grad, g2d) if want_2d else grad


def project_jacobian(scene, cam, g):
    p, stride = _params64(scene)
    P = p.shape[0]
    jac = np.zeros((9, P))
    c = cam_record(cam)
    flags = lib().or_project_jacobian(_p(p), scene["n"], stride, scene["deg"], _p(c), int(g), _p(jac))
    return jac, int(flags)


def gaussian_flags(scene, cam):
    p, stride = _params64(scene)
    f = np.zeros(scene["n"], dtype=np.int32)
    lib().or_gaussian_flags(_p(p), scene["n"], stride, scene["deg"], _p(cam_record(cam)),
                            _p(f, ctypes.c_int))
    return f


def l1(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.ascontiguousarray(y, dtype=np.float64).ravel()
    g = np.zeros_like(x)
    loss = lib().or_l1(_p(x), _p(y), x.size, _p(g))
    return float(loss), g


def adam(p, g, m, v, lr_planes, step, b1=0.9, b2=0.999, eps=1e-15, n=None):
    """In-place FP64 Adam on [P, stride] arrays (float64, C-contiguous)."""
    P, stride = p.shape
    n = stride if n is None else n
    lr = np.ascontiguousarray(lr_planes, dtype=np.float64)
    assert lr.shape == (P,)
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.shape == (P, stride)
    lib().or_adam(_p(p), _p(g), _p(m), _p(v), P, n, stride, _p(lr), b1, b2, eps, int(step))


def adam_visible(p, g, m, v, lr_planes, step, visible, b1=0.9, b2=0.999, eps=1e-15, n=None):
    """In-place FP64 visible-only Adam: Gaussians with visible[i] == 0 keep
    p, m and v; the others take the Adam step."""
    P, stride = p.shape
    n = stride if n is None else n
    lr = np.ascontiguousarray(lr_planes, dtype=np.float64)
    vis = np.ascontiguousarray(np.asarray(visible)[:n], dtype=np.uint8)
    assert lr.shape == (P,) and vis.shape == (n,)
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.shape == (P, stride)
    lib().or_adam_visible(_p(p), _p(g), _p(m), _p(v), P, n, stride, _p(lr), b1, b2, eps, int(step),
                          _p(vis, ctypes.c_uint8))


def visible_in_batch(scene, cams):
    """1 for each Gaussian that touches at least one tile in some view."""
    vis = np.zeros(scene["n"], dtype=np.uint8)
    for cam in cams:
        vis |= (project(scene, cam)["tiles"] > 0).astype(np.uint8)
    return vis


def sh_basis(deg, dirs):
    dirs = np.ascontiguousarray(dirs, dtype=np.float64)
    K = (deg + 1) ** 2
    out = np.zeros((dirs.shape[0], K))
    lib().or_sh_basis(deg, _p(dirs), dirs.shape[0], _p(out))
    return out


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))

"""FP64 adaptive density control of 3D-GS (plain numpy).

TEST INFRASTRUCTURE: only the tests use this module; the product path never
does.

The paper is silent on densification; this is the standard 3D-GS step
written out (the reading the hot-path scope table gives for its NEXT-2 row):

  statistic  per Gaussian, summed over the training views where it touches
             a tile: g_i = sum || (dL/dmu2D_x W / 2, dL/dmu2D_y H / 2) ||
             (the screen-space mean gradient in normalised device
             coordinates) and c_i = the number of such views.
  decide     avg_i = g_i / c_i (0 when c_i = 0); smax_i = max_k exp(s_ik).
             prune:  sigma(o_i) < min_opacity                -> no output
             clone:  avg_i >= tau and smax_i <= dense * extent -> the
                     Gaussian, then a copy with zero Adam moments
             split:  avg_i >= tau and smax_i > dense * extent  -> N = 2 new
                     Gaussians replacing it: mean mu + R(q/|q|) (exp(s) * z_k)
                     with z_k the given standard normals, log-scales
                     s - log(0.8 N), the other parameters copied, zero moments
             else    the Gaussian unchanged.
  order      outputs in input order, a Gaussian's outputs together.
"""
from __future__ import annotations

import math

import numpy as np


def ndc_grad_stat(g2d_views, cams, visible):
    """sum over views of ||(dmu_x W/2, dmu_y H/2)|| where visible[v][i], and
    the view count.  g2d_views: list of [n, >= 2] arrays (dL/dmu2D)."""
    n = g2d_views[0].shape[0]
    s = np.zeros(n)
    c = np.zeros(n)
    for g, cam, vis in zip(g2d_views, cams, visible):
        gx = g[:, 0] * cam["width"] / 2.0
        gy = g[:, 1] * cam["height"] / 2.0
        s += np.where(vis, np.sqrt(gx * gx + gy * gy), 0.0)
        c += vis
    return s, c


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def densify(params, m, v, grad_accum, count, noise, tau=2e-4, dense=0.01, extent=1.0, min_opacity=0.005,
            split_n=2):
    """params, m, v: [P, n]; noise [n, split_n, 3].  Returns (p, m, v) of the
    new set ([P, n_out]) and the per-Gaussian decision (0 prune, 1 keep,
    2 clone, 3 split)."""
    p = np.asarray(params, np.float64)
    P, n = p.shape
    avg = np.where(count > 0, grad_accum / np.maximum(count, 1), 0.0)
    smax = np.exp(p[3:6].max(axis=0))
    opac = 1.0 / (1.0 + np.exp(-p[10]))
    big = avg >= tau
    kind = np.ones(n, np.int64)
    kind[big & (smax <= dense * extent)] = 2
    kind[big & (smax > dense * extent)] = 3
    kind[opac < min_opacity] = 0
    po, mo, vo = [], [], []
    zero = np.zeros(P)
    for i in range(n):
        if kind[i] == 1:
            po.append(p[:, i]); mo.append(m[:, i]); vo.append(v[:, i])
        elif kind[i] == 2:
            po += [p[:, i], p[:, i].copy()]
            mo += [m[:, i], zero]
            vo += [v[:, i], zero]
        elif kind[i] == 3:
            R = _rot(p[6:10, i])
            s = np.exp(p[3:6, i])
            for k in range(split_n):
                q = p[:, i].copy()
                q[0:3] = p[0:3, i] + R @ (s * noise[i, k])
                q[3:6] = p[3:6, i] - math.log(0.8 * split_n)
                po.append(q); mo.append(zero); vo.append(zero)
    if not po:
        return np.zeros((P, 0)), np.zeros((P, 0)), np.zeros((P, 0)), kind
    return np.stack(po, 1), np.stack(mo, 1), np.stack(vo, 1), kind

"""FP64 point-cloud initialisation of the Gaussians (plain numpy / scipy).

TEST INFRASTRUCTURE: only the tests use this module; the product path never
does.

The paper initialises 3D-GS from the isosurface of a volume extracted as a
point cloud (Method Overview: the contour filter's output replaces SfM
points).  Written out here:

  crossings  for every grid vertex (x fastest, then y, then z) and each of
             its +x, +y, +z edges inside the grid whose end values a, b lie
             on different sides of the level (a >= iso differs from
             b >= iso): the point p_a + t (p_b - p_a), t = (iso - a)/(b - a),
             and the normal: the volume gradient (central differences, one-
             sided at the border, as numpy.gradient) interpolated the same
             way and normalised.
  scales     s = log sqrt(mean squared distance to the k = 3 nearest other
             points), the squared mean floored at 1e-14.
  Gaussians  mean = point, log-scales (s, s, s + log(flatten)), rotation
             taking +z onto the normal (quaternion (1 + n_z, -n_y, n_x, 0),
             normalised; (0, 1, 0, 0) when n = -z), opacity logit as given,
             SH DC 2 sqrt(pi) (c - 1/2) with the Lambertian grey
             c = 0.1 + 0.9 max(0, n . (1, 1, 1)/sqrt 3), higher SH 0.
"""
from __future__ import annotations

import math

import numpy as np


def iso_crossings(volume, iso, origin, spacing):
    """volume [nz][ny][nx] (float32 values); returns points [m, 3] and unit
    normals [m, 3] (x, y, z) in the canonical order."""
    f = np.asarray(volume)
    nz, ny, nx = f.shape
    inside = f >= np.float32(iso)
    g = np.gradient(f.astype(np.float64), spacing[2], spacing[1], spacing[0], edge_order=1)  # d/dz, d/dy, d/dx
    grad = np.stack([g[2], g[1], g[0]], axis=-1)  # (gx, gy, gz) per vertex
    pts, nrm = [], []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for (dx, dy, dz) in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    x2, y2, z2 = x + dx, y + dy, z + dz
                    if x2 >= nx or y2 >= ny or z2 >= nz:
                        continue
                    if inside[z, y, x] == inside[z2, y2, x2]:
                        continue
                    a, b = float(f[z, y, x]), float(f[z2, y2, x2])
                    t = (iso - a) / (b - a)
                    pa = np.array([origin[0] + spacing[0] * x, origin[1] + spacing[1] * y, origin[2] + spacing[2] * z])
                    step = np.array([spacing[0] * dx, spacing[1] * dy, spacing[2] * dz])
                    pts.append(pa + t * step)
                    gv = grad[z, y, x] + t * (grad[z2, y2, x2] - grad[z, y, x])
                    nrm.append(gv / np.linalg.norm(gv))
    return np.array(pts).reshape(-1, 3), np.array(nrm).reshape(-1, 3)


def knn_log_scales(points, k=3):
    """0.5 log(max(1e-14, mean of the k smallest squared distances to other
    points)), by scipy's k-d tree (exact nearest neighbours)."""
    from scipy.spatial import cKDTree
    p = np.asarray(points, np.float64)
    d, _ = cKDTree(p).query(p, k=k + 1)
    msq = np.maximum(np.mean(d[:, 1:] ** 2, axis=1), 1e-14)
    return 0.5 * np.log(msq)


def knn_log_scales_brute(points, k=3):
    p = np.asarray(points, np.float64)
    d2 = ((p[:, None, :] - p[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    near = np.sort(d2, axis=1)[:, :k]
    return 0.5 * np.log(np.maximum(near.mean(axis=1), 1e-14))


def init_gaussians(points, normals, flatten=0.3, opacity_logit=2.0, deg=3):
    """Parameter planes [P, n] (float64) of the initial Gaussians."""
    p = np.asarray(points, np.float64)
    nr = np.asarray(normals, np.float64)
    n = p.shape[0]
    s = knn_log_scales(p)
    K = (deg + 1) ** 2
    out = np.zeros((11 + 3 * K, n))
    out[0:3] = p.T
    out[3] = s
    out[4] = s
    out[5] = s + math.log(flatten)
    w = 1.0 + nr[:, 2]
    q = np.stack([w, -nr[:, 1], nr[:, 0], np.zeros(n)], axis=1)
    bad = w < 1e-6
    q[bad] = [0.0, 1.0, 0.0, 0.0]
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    out[6:10] = q.T
    out[10] = opacity_logit
    light = np.ones(3) / math.sqrt(3.0)
    c = 0.1 + 0.9 * np.maximum(0.0, nr @ light)
    dc = (c - 0.5) * 2.0 * math.sqrt(math.pi)
    for ch in range(3):
        out[11 + ch] = dc
    return out
